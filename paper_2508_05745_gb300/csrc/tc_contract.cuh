// Two-site contraction on the tensor cores (mixed precision, sm_103a):
// Theta = A_q A_{q+1} as a (2 dl x dm)(dm x 2 dr) complex GEMM (the
// contraction of Sec. IV.A) in complex FP32, from 3xTF32 split products with
// FP32 accumulation in tensor memory.
//
// The complex GEMM is taken in its real embedding: a complex64 row of A is a
// real row of (re, im) pairs, so with
//   Br'[2k][n] = Re B[k][n], Br'[2k+1][n] = -Im B[k][n],
//   Bi'[2k][n] = Im B[k][n], Bi'[2k+1][n] =  Re B[k][n]
// Re Theta = A_real Br' and Im Theta = A_real Bi'.  Each operand x is split
// into x = hi + lo with hi, lo in tf32, and a real product X Y is taken as
// Xhi Yhi + Xhi Ylo + Xlo Yhi.
//  - A_real needs no rearrangement: TMA tensor copies (cp.async.bulk.tensor,
//    3-D maps over the site slots of all trajectories) write it straight into
//    the 64-byte-swizzled K-major layout that tcgen05.mma reads.  The tensor
//    core reads an FP32 operand as tf32 by dropping its 13 low mantissa bits,
//    so the raw tile is the high part as it stands and only the low part A -
//    trunc(A) is formed, elementwise.
//  - B is split per half of N (128 columns of Theta) into a high and a low
//    plane whose rows are [Br' columns | Bi' columns] (K-major, no swizzle:
//    8 x 16-byte core matrices, LBO = 128 bytes along K, SBO = 512 bytes
//    between 8-row groups), so one MMA of N = 2 x 128 yields Re and Im side by
//    side.  Both M tiles of A share the planes; the accumulators (2 M tiles x
//    256 columns) fill the 512 tensor-memory columns.
//  - Per chunk of 8 complex k: 2 M tiles x 3 products x 2 k-steps = 12
//    tcgen05.mma (kind::tf32) of 128 x 256 x 8.
//
// One CTA of kThreads per trajectory, specialised by warp: warps 0-7 split the
// operands and read the accumulators back (tcgen05.ld 32x32b, staged through
// shared memory into 128-byte row segments); one lane of warp 8 issues the TMA
// copies and the MMAs.  Hand-offs are mbarriers:
//   tma_full[s]   copy of a chunk landed in TMA stage s (kNTma stages)
//   split_full[s] the 256 split threads filled split stage s (2 stages)
//   mma_done[s]   the MMAs that read split stage s finished (tcgen05.commit)
//   acc_empty     the 256 readout threads are done with the accumulators
// Every wait is bounded (about two seconds) and gives up once another thread
// has flagged an error; the issuing lane then waits (bounded) for its copies
// and MMAs still in flight so that the CTA can free its tensor memory, and the
// trajectory is flagged TS_COPY by the caller.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace lemps {
namespace tc {

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

constexpr int kKC = 8;                          // complex k per chunk (16 real: one 64-byte row)
constexpr int kNH = 128;                        // Theta columns per N half
constexpr int kWorkers = 256;                   // split / readout threads (warps 0-7)
constexpr int kThreads = kWorkers + 32;         // + the issuing warp
constexpr int kNTma = 4;                        // TMA stages
constexpr int kAtile = 128 * 64;                // 8 KB: one M tile of A, 128 rows x 64 bytes
constexpr int kAhiBytes = 2 * kAtile;           // both M tiles
constexpr int kBrawBytes = 2 * kKC * 128 * 8;   // 16 KB: rows 2k + s of B, cap <= 128 columns
constexpr int kTmaStage = kAhiBytes + kBrawBytes;              // 32 KB
constexpr int kBplane = (2 * kNH / 8) * 512;                   // 16 KB: 256 rows x 16 real k
constexpr int kSplitStage = kAhiBytes + 2 * kBplane;           // A lo (16 KB) + B hi, lo (32 KB)
constexpr int kOffSplit = kNTma * kTmaStage;                   // 128 KB
constexpr int kSmemBytes = kOffSplit + 2 * kSplitStage + 1024;  // 224 KB + alignment slack
constexpr int kNumBars = kNTma + 5;

// K-major, 64-byte swizzle: 8-row atoms of 512 bytes (SBO), layout type 4
// (the leading byte offset is not used by swizzled K-major layouts).
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// low part of x for the 3xTF32 split when the high part is x with its 13 low
// mantissa bits dropped (how the tensor core reads an FP32 operand)
__device__ __forceinline__ float lo_of_trunc(float x) {
  const float hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  return __uint_as_float(to_tf32(x - hi));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok)
               : "r"(smem_addr(bar)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// L2 prefetch of bytes (a multiple of 16) from a 16-byte-aligned address, in
// pieces of at most 32 KB.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (uint32_t o = 0; o < bytes; o += 32768u) {
    const uint32_t n = min(32768u, bytes - o);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + o), "r"(n) : "memory");
  }
}
// Bounded wait that also gives up once *err is set; a timeout sets *err.
__device__ __forceinline__ bool wait_or_err(uint64_t* bar, uint32_t parity, volatile int* err) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*err) return false;
    if (clock64() - t0 > (1LL << 32)) {
      *err = 1;
      return false;
    }
  }
}

// Initialises the kNumBars mbarriers of gemm (one thread, before the CTA
// synchronises).
__device__ __forceinline__ void init_bars(uint64_t* bars) {
  for (int i = 0; i < kNTma; ++i) mbar_init(&bars[i], 1);
  mbar_init(&bars[kNTma + 0], kWorkers);   // split_full
  mbar_init(&bars[kNTma + 1], kWorkers);
  mbar_init(&bars[kNTma + 2], 1);          // mma_done
  mbar_init(&bars[kNTma + 3], 1);
  mbar_init(&bars[kNTma + 4], kWorkers);   // acc_empty
}

// Theta (M x N = 2 dr, row-major, ldc even, C 16-byte aligned; M <= 256,
// N <= 256) = A B for one trajectory t: A from the A map (site q as [2 cap_q][cap_{q+1}] complex64,
// box 8 x 128, 64-byte swizzle), B from the B map (site q + 1 as [2
// cap_{q+1}][cap_{q+2}], box cap_{q+2} x 16; cap_{q+2} <= 128 and even);
// a_slot, b_slot: the same two site slots of trajectory t (capm = cap_{q+1}
// columns of A; their first M and 2 K rows are prefetched into L2 at the start
// of each half of N, ahead of the tile copies).  Called by all kThreads threads
// once per CTA; bars: kNumBars mbarriers initialised by init_bars; tmem: the
// 512-column allocation; err: a shared int set to 0.  Returns false on a
// timeout (uniform over the CTA).
__device__ __noinline__ bool gemm(const CUtensorMap* mapA, const CUtensorMap* mapB, int t, int M, int K, int dr,
                                  int capr, const cpx<float>* a_slot, int capm, const cpx<float>* b_slot,
                                  unsigned char* sm, uint64_t* bars, uint32_t tmem, cpx<float>* C, int ldc,
                                  volatile int* err) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = 2 * dr, nhalf = (N + kNH - 1) / kNH;
  const int nchunk = (K + kKC - 1) / kKC, G = nhalf * nchunk;
  const int nmt = (M + 127) / 128;              // M tiles (1 or 2)
  uint64_t* tma_full = bars;
  uint64_t* split_full = bars + kNTma;
  uint64_t* mma_done = bars + kNTma + 2;
  uint64_t* acc_empty = bars + kNTma + 4;
  if (warp == kWorkers / 32) {
    // ---- issuing lane: TMA copies and MMAs ----
    if (lane == 0) {
      const uint32_t sbase = smem_addr(sm);
      const uint32_t abytes = (uint32_t)(nmt * kAtile), bbytes = (uint32_t)(2 * kKC * capr * 8);
      auto issue_tma = [&](int x) {                // chunk x (K chunk x % nchunk) into stage x % kNTma
        const int st = x % kNTma, c = x % nchunk;
        if (c == 0) {                              // first chunk of a half: operands into L2
          prefetch_l2(a_slot, (uint32_t)M * (uint32_t)capm * 8u);
          prefetch_l2(b_slot, (uint32_t)(2 * K) * (uint32_t)capr * 8u);
        }
        unsigned char* dst = sm + st * kTmaStage;
        mbar_expect_tx(&tma_full[st], abytes + bbytes);
        for (int mt = 0; mt < nmt; ++mt) tma_load_3d(dst + mt * kAtile, mapA, c * kKC, mt * 128, t, &tma_full[st]);
        tma_load_3d(dst + kAhiBytes, mapB, 0, 2 * c * kKC, t, &tma_full[st]);
      };
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      int issued = 0, committed = 0;
      for (; issued < G && issued < kNTma - 1; ++issued) issue_tma(issued);
      for (int g = 0; g < G; ++g) {
        const int h = g / nchunk, c = g - h * nchunk;
        if (c == 0 && h > 0 && !wait_or_err(acc_empty, (uint32_t)((h - 1) & 1), err)) break;
        if (!wait_or_err(&split_full[g & 1], (uint32_t)((g >> 1) & 1), err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int nh = min(kNH, N - h * kNH), nhp = (nh + 15) & ~15;
        const uint32_t idesc = idesc_tf32(128, 2 * nhp, false);
        const uint32_t sA = sbase + (uint32_t)((g % kNTma) * kTmaStage);
        const uint32_t sAl = sbase + (uint32_t)(kOffSplit + (g & 1) * kSplitStage);
        const uint32_t sBh = sAl + (uint32_t)kAhiBytes, sBl = sBh + (uint32_t)kBplane;
        for (int mt = 0; mt < nmt; ++mt) {
          const uint32_t d = tmem + (uint32_t)(mt * 256);
#pragma unroll
          for (int s = 0; s < 2; ++s) {              // two k-steps of 8 real k (32 bytes)
            const uint64_t ah = desc_sw64(sA + mt * kAtile + s * 32), al = desc_sw64(sAl + mt * kAtile + s * 32);
            const uint64_t bh = smem_desc(sBh + s * 256, 128, 512), bl = smem_desc(sBl + s * 256, 128, 512);
            mma_tf32(d, ah, bh, idesc, (c > 0 || s > 0) ? 1u : 0u);
            mma_tf32(d, ah, bl, idesc, 1u);
            mma_tf32(d, al, bh, idesc, 1u);
          }
        }
        mma_commit(&mma_done[g & 1]);
        committed = g + 1;
        // the stage of chunk g - 1 takes chunk g + kNTma - 1 once its MMAs are done
        if (g >= 1 && !wait_or_err(&mma_done[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1), err)) break;
        if (issued < G) issue_tma(issued++);
      }
      // drain whatever is still in flight (bounded waits that do not give up on *err)
      if (committed > 0) mbar_wait(&mma_done[(committed - 1) & 1], (uint32_t)(((committed - 1) >> 1) & 1));
      for (int x = max(0, issued - kNTma); x < issued; ++x) mbar_wait(&tma_full[x % kNTma], (uint32_t)((x / kNTma) & 1));
    }
    __syncwarp();
  } else {
    // ---- warps 0-7: operand split and accumulator readout ----
    int g = 0;
    bool ok = true;
    for (int h = 0; h < nhalf && ok; ++h) {
      const int n0 = h * kNH, nh = min(kNH, N - n0), nhp = (nh + 15) & ~15;
      if (h > 0 && !wait_or_err(acc_empty, (uint32_t)((h - 1) & 1), err)) break;   // staging reuse
      for (int c = 0; c < nchunk; ++c, ++g) {
        unsigned char* tst = sm + (g % kNTma) * kTmaStage;
        unsigned char* sst = sm + kOffSplit + (g & 1) * kSplitStage;
        if (!wait_or_err(&tma_full[g % kNTma], (uint32_t)((g / kNTma) & 1), err) ||
            (g >= 2 && !wait_or_err(&mma_done[g & 1], (uint32_t)(((g - 2) >> 1) & 1), err))) {
          ok = false;
          break;
        }
        // A low parts, elementwise over the swizzled tiles; entries with
        // complex k >= K (stale slot columns beyond the bond dimension) are
        // zeroed in both parts.  Rows beyond M only feed output rows that are
        // not stored.  In a 64-byte-swizzled tile the 16-byte chunk at
        // position p of row r holds logical chunk p ^ ((r >> 1) & 3), i.e.
        // complex k0 + 2j and k0 + 2j + 1.
        const int k0 = c * kKC;
        {
          float4* hi = reinterpret_cast<float4*>(tst);
          float4* dst = reinterpret_cast<float4*>(sst);
          const bool ragged = k0 + kKC > K;
          for (int e = tid; e < nmt * kAtile / 16; e += kWorkers) {
            float4 x = hi[e];
            if (ragged) {
              const int r = e >> 2, j = (e & 3) ^ ((r >> 1) & 3);
              const int kc = k0 + 2 * j;
              if (kc >= K) x.x = x.y = 0.f;
              if (kc + 1 >= K) {
                x.z = x.w = 0.f;
                hi[e] = x;
              }
            }
            x.x = lo_of_trunc(x.x); x.y = lo_of_trunc(x.y);
            x.z = lo_of_trunc(x.z); x.w = lo_of_trunc(x.w);
            dst[e] = x;
          }
        }
        // B planes of this half, K-major without swizzle: row n < nhp holds
        // Br' column n0 + n, row nhp + n holds Bi' column n0 + n.  A warp
        // covers 8 n x 4 k, which spreads its 8-byte stores over all banks.
        {
          const cpx<float>* braw = reinterpret_cast<const cpx<float>*>(tst + kAhiBytes);
          unsigned char* bh = sst + kAhiBytes;
          unsigned char* bl = bh + kBplane;
          for (int e = tid; e < nhp * kKC; e += kWorkers) {
            const int n = ((e >> 6) << 3) | (e & 7), kk = (e >> 3) & 7;
            const int j = n0 + n;
            cpx<float> x = mk(0.f, 0.f);
            if (n < nh && k0 + kk < K) {
              const int s2 = j >= dr, b = j - s2 * dr;
              x = braw[(2 * kk + s2) * capr + b];
            }
            const float rh = __uint_as_float(to_tf32(x.re)), ih = __uint_as_float(to_tf32(x.im));
            const float rl = __uint_as_float(to_tf32(x.re - rh)), il = __uint_as_float(to_tf32(x.im - ih));
            const uint32_t o = kmajor_off(n, 2 * kk), oi = kmajor_off(nhp + n, 2 * kk);
            *reinterpret_cast<float2*>(bh + o) = make_float2(rh, -ih);    // Br' high
            *reinterpret_cast<float2*>(bh + oi) = make_float2(ih, rh);    // Bi' high
            *reinterpret_cast<float2*>(bl + o) = make_float2(rl, -il);    // Br' low
            *reinterpret_cast<float2*>(bl + oi) = make_float2(il, rl);    // Bi' low
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&split_full[g & 1]);
      }
      if (!ok || !wait_or_err(&mma_done[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1), err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // readout: warp w reads tensor-memory lanes 32 (w % 4) .. of M tile w / 4
      // (row = lane), stages each 32-row x 16-column block in its own 4 KB of
      // the (idle) split stages with 16-byte chunks XOR-swizzled by row, and
      // stores it as 128-byte row segments.
      {
        const int mt = warp >> 2, rbase = mt * 128 + 32 * (warp & 3);
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        float4* stg = reinterpret_cast<float4*>(sm + kOffSplit + warp * 4096);
        if (mt < nmt && rbase < M) {
          for (int c0 = 0; c0 < nhp; c0 += 16) {
            float re[16], im[16];
            ld_32x32b_x16(tmem + lane_base + (uint32_t)(mt * 256 + c0), re);
            ld_32x32b_x16(tmem + lane_base + (uint32_t)(mt * 256 + nhp + c0), im);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q)
              stg[lane * 8 + (q ^ (lane & 7))] = make_float4(re[2 * q], im[2 * q], re[2 * q + 1], im[2 * q + 1]);
            __syncwarp();
#pragma unroll
            for (int it = 0; it < 8; ++it) {
              const int rr = it * 4 + (lane >> 3), q = lane & 7, row = rbase + rr, col = n0 + c0 + 2 * q;
              const float4 v = stg[rr * 8 + (q ^ (rr & 7))];
              if (row < M) {
                if (c0 + 2 * q + 1 < nh) *reinterpret_cast<float4*>(C + (int64_t)row * ldc + col) = v;
                else if (c0 + 2 * q < nh) C[(int64_t)row * ldc + col] = mk(v.x, v.y);
              }
            }
            __syncwarp();
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acc_empty);
    }
  }
  __syncthreads();
  return *err == 0;
}

}  // namespace tc
}  // namespace lemps
