// Shared device helpers: complex arithmetic templated on the real type,
// Philox4x64-10, reductions and the per-simulation device context.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace lemps {

template <class R>
struct alignas(2 * sizeof(R)) cpx {
  R re, im;
};

template <class R> __host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { cpx<R> z; z.re = a; z.im = b; return z; }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return mk(-a.re, -a.im); }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> __host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return mk(s * a.re, s * a.im); }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, R s) { return mk(s * a.re, s * a.im); }
template <class R> __host__ __device__ __forceinline__ cpx<R>& operator+=(cpx<R>& a, cpx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> __host__ __device__ __forceinline__ cpx<R>& operator-=(cpx<R>& a, cpx<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <class R> __host__ __device__ __forceinline__ cpx<R> conj(cpx<R> a) { return mk(a.re, -a.im); }
template <class R> __host__ __device__ __forceinline__ R norm2(cpx<R> a) { return a.re * a.re + a.im * a.im; }
// conj(a) * b
template <class R> __host__ __device__ __forceinline__ cpx<R> cdot(cpx<R> a, cpx<R> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// acc += a * b
template <class R> __host__ __device__ __forceinline__ void cfma(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <class R> __host__ __device__ __forceinline__ void cfmac(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <class D, class S> __host__ __device__ __forceinline__ cpx<D> cast(cpx<S> a) { return mk<D>((D)a.re, (D)a.im); }

typedef cpx<double> zd;
typedef cpx<float> zf;

// ---- Philox4x64-10 (Salmon et al., SC'11) ------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

constexpr uint64_t kDomainTrajectory = 0x4C454D5053545241ULL;

__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t traj, uint64_t gate, uint64_t slot) {
  uint64_t c[4] = {traj, gate, slot, 0ULL};
  philox4x64_10(c, seed, kDomainTrajectory);
  return (double)(c[0] >> 11) * (1.0 / 9007199254740992.0);
}

// ---- status codes written per trajectory ------------------------------------
enum TrajStatus : int32_t {
  TS_OK = 0,
  TS_NAN = 1,        // NaN / Inf in a reduced density or branch weight
  TS_NORM = 2,       // two-site tensor lost its norm
  TS_JACOBI = 4,     // eigensolver hit its sweep cap above tolerance
  TS_SHAPE = 8,      // bond dimensions outside capacity (internal error)
  TS_COPY = 16       // an asynchronous copy missed its time limit (internal error)
};

// ---- mbarrier and 1-D bulk copies (TMA engine) ------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes barrier initialization, and this thread's earlier generic-proxy
// writes (shared or global), visible to later bulk copies.
__device__ __forceinline__ void fence_for_bulk_copies() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) that completes its byte count on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Waits for the phase of parity `parity` of `bar` to complete; gives up and
// returns false after about two seconds (2^32 SM cycles).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1LL << 32)) return false;
  }
}

// ---- block reductions ---------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums NV (2, 4, 8, 16 or 32) per-lane values over the warp at once: log2(NV)
// halving rounds of a reduce-scatter butterfly, then plain rounds over the
// remaining lane bits.  Returns the total of value Scatter<NV>::index(lane)
// (the lane's top log2(NV) bits, 4 first, spell it from its most significant
// bit down; for NV = 32 that is the lane itself); d is clobbered.  Costs NV + 4 - log2(NV) shuffles instead of 5 NV.
template <int NV>
struct Scatter {
  static constexpr int LG = NV == 32 ? 5 : (NV == 16 ? 4 : (NV == 8 ? 3 : (NV == 4 ? 2 : 1)));
  __device__ __forceinline__ static int index(int lane) {
    int e = 0;
#pragma unroll
    for (int r = 0; r < LG; ++r) e = (e << 1) | ((lane >> (4 - r)) & 1);
    return e;
  }
  // first lane that holds the total of value e
  __device__ __forceinline__ static int source(int e) {
    int src = 0;
#pragma unroll
    for (int r = 0; r < LG; ++r)
      if (e & (1 << (LG - 1 - r))) src |= 16 >> r;
    return src;
  }
};
template <int NV, class T>
__device__ __forceinline__ T warp_reduce_scatter(T (&d)[NV], int lane) {
  constexpr int LG = Scatter<NV>::LG;
#pragma unroll
  for (int r = 0; r < LG; ++r) {
    const int s = 16 >> r;
    const int h = NV >> (r + 1);
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const T send = up ? d[k] : d[k + h];
      const T keepv = up ? d[k + h] : d[k];
      d[k] = keepv + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  T tot = d[0];
#pragma unroll
  for (int r = LG; r < 5; ++r) tot += __shfl_xor_sync(0xffffffffu, tot, 16 >> r);
  return tot;
}

// Sum over the block; every thread receives the result.  `scratch` holds at
// least blockDim.x/32 values.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  return s;
}

}  // namespace lemps
