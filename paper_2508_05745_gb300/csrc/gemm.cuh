// CTA-level complex GEMM through shared memory (SIMT, FP32 or FP64), used by
// the per-trajectory kernels: C[M x N] = sum_k A(i, k) B(k, j).
//
// Output tiles of BM x BN (default 64 x 64) and K slabs of 16 over 256
// threads; each thread owns a (BM/16) x (BN/16) micro-tile interleaved with
// stride 16 in both dimensions, so shared-memory reads are conflict-free.
// Every output entry is accumulated over k = 0, 1, ..., K-1 in that order
// whatever the tile shape, so all shapes give bit-identical results (which
// lets an autotuner pick the shape per problem size without changing any
// output).  Operands are read through functors (index maps, conjugation,
// padding) and the result is handed to a store functor, which lets kernels
// fuse their epilogues (residual norms, scaling, scatter into site slots).
// A_KFAST / B_KFAST choose the tile-load order so that the underlying memory
// is read along its contiguous dimension.
#pragma once

#include "common.cuh"

namespace lemps {

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 256;

// The tile shapes the autotuner chooses from, per storage precision (index
// 0 is the default).  Complex64 adds rectangular 128-wide register tiles:
// with one CTA per trajectory and few CTAs per SM the kernels are
// latency-bound, and a thread with more independent accumulators hides more
// of it (a 128 x 128 tile would spill: 128 accumulator registers plus the
// prefetched slab).  Complex128 adds narrower tiles instead (its 128-wide
// tiles would need 256 accumulator registers per thread).  The 32 x 32 tile
// wastes the least on small and ragged bond dimensions.
constexpr int kNumGemmTiles = 4;
template <class R, int ID> struct GemmTileShape;
template <> struct GemmTileShape<float, 0> { static constexpr int BM = 64, BN = 64; };
template <> struct GemmTileShape<float, 1> { static constexpr int BM = 128, BN = 64; };
template <> struct GemmTileShape<float, 2> { static constexpr int BM = 64, BN = 128; };
template <> struct GemmTileShape<float, 3> { static constexpr int BM = 32, BN = 32; };
template <> struct GemmTileShape<double, 0> { static constexpr int BM = 64, BN = 64; };
template <> struct GemmTileShape<double, 1> { static constexpr int BM = 32, BN = 64; };
template <> struct GemmTileShape<double, 2> { static constexpr int BM = 64, BN = 32; };
template <> struct GemmTileShape<double, 3> { static constexpr int BM = 32, BN = 32; };

// Rows are padded by one element: a tile loaded with k fastest (A_KFAST /
// B_KFAST) stores 16 consecutive k of one column per half-warp, which would hit
// one bank group at a stride of 64 elements; at 65 they fall on distinct banks.
// The multiply reads (fixed k, consecutive i or j) stay conflict-free.
template <class R, int BM = kGemmBM, int BN = kGemmBN>
struct GemmSmem {
  cpx<R> a[kGemmBK][BM + 1];
  cpx<R> b[kGemmBK][BN + 1];
};

template <class R, bool A_KFAST, bool B_KFAST, int BM, int BN, class FA, class FB, class FC>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, FA loadA, FB loadB, FC store, GemmSmem<R, BM, BN>& sm,
                                         bool upper_only = false) {
  static_assert(BM % 16 == 0 && BN % 16 == 0, "tile sides are multiples of the 16 x 16 thread grid");
  constexpr int TM = BM / 16, TN = BN / 16;   // micro-tile of a thread
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int i0 = 0; i0 < M; i0 += BM) {
    for (int j0 = 0; j0 < N; j0 += BN) {
      if (upper_only && j0 + BN <= i0) continue;  // tile strictly below the diagonal
      cpx<R> acc[TM][TN];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = mk<R>(0, 0);
      // the next K slab is loaded into registers while the current one is
      // multiplied out of shared memory
      constexpr int LA = BM * kGemmBK / kGemmThreads, LB = kGemmBK * BN / kGemmThreads;
      cpx<R> ra[LA], rb[LB];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < LA; ++q) {
          const int e = tid + q * kGemmThreads;
          int i, k;
          if (A_KFAST) { i = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / BM; i = e % BM; }
          ra[q] = (i0 + i < M && k0 + k < K) ? loadA(i0 + i, k0 + k) : mk<R>(0, 0);
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          const int e = tid + q * kGemmThreads;
          int k, j;
          if (B_KFAST) { j = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / BN; j = e % BN; }
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
          else { k = e / BM; i = e % BM; }
          sm.a[k][i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          const int e = tid + q * kGemmThreads;
          int k, j;
          if (B_KFAST) { j = e / kGemmBK; k = e % kGemmBK; }
          else { k = e / BN; j = e % BN; }
          sm.b[k][j] = rb[q];
        }
        __syncthreads();
        if (k0 + kGemmBK < K) fetch(k0 + kGemmBK);
#pragma unroll
        for (int k = 0; k < kGemmBK; ++k) {
          cpx<R> av[TM], bv[TN];
#pragma unroll
          for (int r = 0; r < TM; ++r) av[r] = sm.a[k][ty + 16 * r];
#pragma unroll
          for (int c = 0; c < TN; ++c) bv[c] = sm.b[k][tx + 16 * c];
#pragma unroll
          for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) cfma(acc[r][c], av[r], bv[c]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
          const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
          if (i < M && j < N) store(i, j, acc[r][c]);
        }
    }
  }
}

}  // namespace lemps
