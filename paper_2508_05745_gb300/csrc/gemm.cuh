// CTA-level complex GEMM through shared memory (SIMT, FP32 or FP64), used by
// the per-trajectory kernels: C[M x N] = sum_k A(i, k) B(k, j).
//
// Tiles of 64 x 64 x 16 over 256 threads; each thread owns a 4 x 4 micro-tile
// interleaved with stride 16 in both dimensions, so shared-memory reads are
// conflict-free.  Operands are read through functors (index maps, conjugation,
// padding) and the result is handed to a store functor, which lets kernels
// fuse their epilogues (residual norms, scaling, scatter into site slots).
// A_KFAST / B_KFAST choose the tile-load order so that the underlying memory
// is read along its contiguous dimension.
#pragma once

#include "common.cuh"

namespace lemps {

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 256;

// Rows are padded by one element: a tile loaded with k fastest (A_KFAST /
// B_KFAST) stores 16 consecutive k of one column per half-warp, which would hit
// one bank group at a stride of 64 elements; at 65 they fall on distinct banks.
// The multiply reads (fixed k, consecutive i or j) stay conflict-free.
template <class R>
struct GemmSmem {
  cpx<R> a[kGemmBK][kGemmBM + 1];
  cpx<R> b[kGemmBK][kGemmBN + 1];
};

template <class R, bool A_KFAST, bool B_KFAST, class FA, class FB, class FC>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, FA loadA, FB loadB, FC store, GemmSmem<R>& sm,
                                         bool upper_only = false) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int i0 = 0; i0 < M; i0 += kGemmBM) {
    for (int j0 = 0; j0 < N; j0 += kGemmBN) {
      if (upper_only && j0 + kGemmBN <= i0) continue;  // tile strictly below the diagonal
      cpx<R> acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = mk<R>(0, 0);
      // the next K slab is loaded into registers while the current one is
      // multiplied out of shared memory
      constexpr int LA = kGemmBM * kGemmBK / kGemmThreads, LB = kGemmBK * kGemmBN / kGemmThreads;
      cpx<R> ra[LA], rb[LB];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < LA; ++q) {
          const int e = tid + q * kGemmThreads;
          int i, k;
          if (A_KFAST) { i = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / kGemmBM; i = e % kGemmBM; }
          ra[q] = (i0 + i < M && k0 + k < K) ? loadA(i0 + i, k0 + k) : mk<R>(0, 0);
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          const int e = tid + q * kGemmThreads;
          int k, j;
          if (B_KFAST) { j = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / kGemmBN; j = e % kGemmBN; }
          rb[q] = (j0 + j < N && k0 + k < K) ? loadB(k0 + k, j0 + j) : mk<R>(0, 0);
        }
      };
      if (K > 0) fetch(0);
      for (int k0 = 0; k0 < K; k0 += kGemmBK) {
#pragma unroll
        for (int q = 0; q < LA; ++q) {
          const int e = tid + q * kGemmThreads;
          int i, k;
          if (A_KFAST) { i = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / kGemmBM; i = e % kGemmBM; }
          sm.a[k][i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          const int e = tid + q * kGemmThreads;
          int k, j;
          if (B_KFAST) { j = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / kGemmBN; j = e % kGemmBN; }
          sm.b[k][j] = rb[q];
        }
        __syncthreads();
        if (k0 + kGemmBK < K) fetch(k0 + kGemmBK);
#pragma unroll
        for (int k = 0; k < kGemmBK; ++k) {
          cpx<R> av[4], bv[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) av[r] = sm.a[k][ty + 16 * r];
#pragma unroll
          for (int c = 0; c < 4; ++c) bv[c] = sm.b[k][tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) cfma(acc[r][c], av[r], bv[c]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
          if (i < M && j < N) store(i, j, acc[r][c]);
        }
    }
  }
}

}  // namespace lemps
