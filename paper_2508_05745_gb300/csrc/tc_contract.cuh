// Two-site contraction on the tensor cores (mixed precision, sm_103a):
// Theta = A_q A_{q+1} as a (2 dl x dm)(dm x 2 dr) complex GEMM, complex FP32
// built from 3xTF32 split products with FP32 accumulation in tensor memory
// (the contraction of Sec. IV.A; the path's precision pattern for the
// contractions).  Each complex64 operand x is split into tf32 parts x = hi +
// lo (hi = x rounded to tf32, lo = the rest rounded to tf32), and a real
// product X Y is taken as Xhi Yhi + Xhi Ylo + Xlo Yhi, so
//   Re Theta = Ar Br - Ai Bi,   Im Theta = Ar Bi + Ai Br
// takes 12 tcgen05.mma (kind::tf32, M = 128, N = 2 dr rounded up to 16, K = 8)
// per 8 columns of A; the minus sign is the MMA's negate-A bit.
//
// Data flow per trajectory (one CTA of 256 threads; at most one CTA per SM):
//  - the raw complex64 tiles of A (128 rows x 16 k) and of B (32 rows (2k + s)
//    x cap columns) are fetched by TMA tensor copies (cp.async.bulk.tensor,
//    3-D maps over the site slots of all trajectories) onto an mbarrier;
//  - the threads split them into hi/lo tf32 planes of Re and Im in the
//    canonical K-major layout without swizzle (8 x 16-byte core matrices;
//    LBO = 128 bytes between core matrices along K, SBO = 512 bytes between
//    8-row groups), zeroing the rows and columns beyond the actual bond
//    dimensions;
//  - one thread issues the MMAs into two accumulators in tensor memory (Re at
//    column 0, Im at column 256; 512 columns allocated) and commits them to an
//    mbarrier;
//  - after the last K chunk the accumulators are read back (tcgen05.ld
//    32x32b) and Theta is stored to the two-site workspace.
// Every mbarrier wait is bounded (about two seconds) and its outcome is agreed
// by the whole CTA; on a timeout the operations in flight get a second bounded
// wait, the trajectory is flagged TS_COPY, and the CTA frees its tensor memory
// and returns.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace lemps {
namespace tc {

constexpr int kKC = 16;            // columns of A (rows of B) per chunk
constexpr int kM = 128;            // MMA M (one M tile)
constexpr int kNmax = 256;         // MMA N limit: 2 dr <= 256
constexpr int kThreads = 256;

// Shared-memory layout (bytes from a 1024-aligned base).
constexpr int kArawBytes = kM * kKC * 8;                  // 16 KB: A tile, complex64
constexpr int kBrawBytes = 2 * kKC * 128 * 8;             // 32 KB: B tile, 32 rows x cap (<= 128) complex64
constexpr int kAopBytes = (kM / 8) * 512;                 // 8 KB per tf32 plane of A (16 row groups)
constexpr int kBopBytes = (kNmax / 8) * 512;              // 16 KB per tf32 plane of B^T (32 row groups)
constexpr int kOffAraw = 0;
constexpr int kOffBraw = kOffAraw + kArawBytes;
constexpr int kOffAop = kOffBraw + kBrawBytes;            // 4 planes: Re hi, Re lo, Im hi, Im lo
constexpr int kOffBop = kOffAop + 4 * kAopBytes;          // 4 planes: Re hi, Re lo, Im hi, Im lo
constexpr int kSmemBytes = kOffBop + 4 * kBopBytes + 1024;   // + alignment slack

// Byte offset of element (row r, k) of a K-major tile without swizzle: 8-row
// groups 512 bytes apart (SBO), 16-byte core-matrix columns 128 bytes apart
// (LBO), rows of a core matrix 16 bytes apart.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
  return (uint32_t)((r >> 3) * 512 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// tcgen05 shared-memory matrix descriptor: start address >> 4 (bits 0-13),
// leading byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), version
// 1 (46-47), base offset 0, layout: no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B in
// tf32 (bits 7-9 and 10-12 = 2), optional negation of A (bit 13), both
// operands K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n, bool neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void ld_32x32b_x16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// C[i][j] (i < M, j < N), row-major with leading dimension ldc, = A B with
// A[i][k] = sA[(m0 + i) * lda + k] (rows m0..m0+127 of the A map's tile) and
// B[k][j] = the B map's row 2k + s, column b for j = s * dr + b.  Both maps
// are 3-D over (column, row, trajectory t).  Returns false on a timeout.
// Called by all 256 threads; tmem holds the 512-column allocation.
__device__ __forceinline__ bool gemm_tile(const CUtensorMap* mapA, const CUtensorMap* mapB, int t, int m0, int M,
                                          int K, int dr, int capr, unsigned char* sm, uint64_t* bars,
                                          uint32_t* phase, uint32_t tmem, cpx<float>* C, int ldc) {
  const int tid = threadIdx.x;
  const int N = 2 * dr, Npad = (N + 15) & ~15;
  const cpx<float>* Araw = reinterpret_cast<const cpx<float>*>(sm + kOffAraw);
  const cpx<float>* Braw = reinterpret_cast<const cpx<float>*>(sm + kOffBraw);
  unsigned char* Aop = sm + kOffAop;
  unsigned char* Bop = sm + kOffBop;
  const uint32_t sAop = smem_addr(Aop), sBop = smem_addr(Bop);
  const uint32_t id_pos = idesc_tf32(kM, Npad, false), id_neg = idesc_tf32(kM, Npad, true);
  const int nchunk = (K + kKC - 1) / kKC;
  for (int c = 0; c < nchunk; ++c) {
    const int k0 = c * kKC;
    if (tid == 0) {
      // the raw tiles were last read by the threads (generic proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bars[0], (uint32_t)(kArawBytes + 2 * kKC * capr * 8));
      tma_load_3d(sm + kOffAraw, mapA, k0, m0, t, &bars[0]);
      tma_load_3d(sm + kOffBraw, mapB, 0, 2 * k0, t, &bars[0]);
    }
    if (!__syncthreads_and(mbar_wait(&bars[0], phase[0]))) {
      // a copy missed its time limit: give it a second bounded wait before the
      // shared memory is given up
      if (tid == 0) mbar_wait(&bars[0], phase[0]);
      __syncthreads();
      return false;
    }
    phase[0] ^= 1u;
    // split into hi/lo tf32 planes, K-major, zero beyond the bond dimensions
    for (int e = tid; e < kM * kKC; e += kThreads) {
      const int i = e / kKC, k = e % kKC;
      cpx<float> x = mk(0.f, 0.f);
      if (m0 + i < M && k0 + k < K) x = Araw[i * kKC + k];
      const uint32_t rh = to_tf32(x.re), ih = to_tf32(x.im);
      const uint32_t rl = to_tf32(x.re - __uint_as_float(rh)), il = to_tf32(x.im - __uint_as_float(ih));
      const uint32_t o = kmajor_off(i, k);
      *reinterpret_cast<uint32_t*>(Aop + 0 * kAopBytes + o) = rh;
      *reinterpret_cast<uint32_t*>(Aop + 1 * kAopBytes + o) = rl;
      *reinterpret_cast<uint32_t*>(Aop + 2 * kAopBytes + o) = ih;
      *reinterpret_cast<uint32_t*>(Aop + 3 * kAopBytes + o) = il;
    }
    for (int e = tid; e < Npad * kKC; e += kThreads) {
      const int j = e / kKC, k = e % kKC;
      cpx<float> x = mk(0.f, 0.f);
      if (j < N && k0 + k < K) {
        const int s2 = j >= dr, b = j - s2 * dr;
        x = Braw[(2 * k + s2) * capr + b];
      }
      const uint32_t rh = to_tf32(x.re), ih = to_tf32(x.im);
      const uint32_t rl = to_tf32(x.re - __uint_as_float(rh)), il = to_tf32(x.im - __uint_as_float(ih));
      const uint32_t o = kmajor_off(j, k);
      *reinterpret_cast<uint32_t*>(Bop + 0 * kBopBytes + o) = rh;
      *reinterpret_cast<uint32_t*>(Bop + 1 * kBopBytes + o) = rl;
      *reinterpret_cast<uint32_t*>(Bop + 2 * kBopBytes + o) = ih;
      *reinterpret_cast<uint32_t*>(Bop + 3 * kBopBytes + o) = il;
    }
    // the planes were written by the generic proxy and are read by the MMA
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dre = tmem, dim = tmem + 256;
#pragma unroll
      for (int s = 0; s < kKC / 8; ++s) {
        auto A = [&](int p) { return smem_desc(sAop + p * kAopBytes + s * 256, 128, 512); };
        auto B = [&](int p) { return smem_desc(sBop + p * kBopBytes + s * 256, 128, 512); };
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        // Re: Ar Br - Ai Bi (3xTF32 each)
        mma_tf32(dre, A(0), B(0), id_pos, acc);
        mma_tf32(dre, A(0), B(1), id_pos, 1u);
        mma_tf32(dre, A(1), B(0), id_pos, 1u);
        mma_tf32(dre, A(2), B(2), id_neg, 1u);
        mma_tf32(dre, A(2), B(3), id_neg, 1u);
        mma_tf32(dre, A(3), B(2), id_neg, 1u);
        // Im: Ar Bi + Ai Br
        mma_tf32(dim, A(0), B(2), id_pos, acc);
        mma_tf32(dim, A(0), B(3), id_pos, 1u);
        mma_tf32(dim, A(1), B(2), id_pos, 1u);
        mma_tf32(dim, A(2), B(0), id_pos, 1u);
        mma_tf32(dim, A(2), B(1), id_pos, 1u);
        mma_tf32(dim, A(3), B(0), id_pos, 1u);
      }
      mma_commit(&bars[1]);
    }
    // the planes and raw tiles are reused by the next chunk: wait for the MMAs
    if (!__syncthreads_and(mbar_wait(&bars[1], phase[1]))) {
      if (tid == 0) mbar_wait(&bars[1], phase[1]);   // MMAs still in flight: bounded wait
      __syncthreads();
      return false;
    }
    phase[1] ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // read the accumulators back: warp w reads TMEM lanes 32 (w % 4) ..,
  // columns of half w / 4
  const int warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane, half = warp >> 2;
  const int ncols = Npad / 2;   // a multiple of 8; read in 16s (the last may overhang into padding)
  for (int c0 = half * ncols; c0 < (half + 1) * ncols; c0 += 16) {
    float re[16], im[16];
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    ld_32x32b_x16(tmem + lane_base + (uint32_t)c0, re);
    ld_32x32b_x16(tmem + lane_base + 256u + (uint32_t)c0, im);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int i = m0 + row;
    if (i < M) {
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = c0 + jj;
        if (j < N && j < (half + 1) * ncols) C[(int64_t)i * ldc + j] = mk(re[jj], im[jj]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  return true;
}

}  // namespace tc
}  // namespace lemps
