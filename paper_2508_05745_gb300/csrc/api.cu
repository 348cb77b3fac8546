// C ABI of the library (include/lemps.h): device allocation, layer
// orchestration and the measure/export calls.  All arithmetic runs in the
// kernels of mps_kernels.cuh and unravel.cuh; the host only schedules them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lemps.h"
#include "big_kernels.cuh"
#include "mps_kernels.cuh"
#include "unravel_iface.h"

using namespace lemps;

namespace {

thread_local std::string g_err;

lemps_status fail(lemps_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

constexpr int kThreads = 256;

}  // namespace

// Layers whose error contributions are kept per trajectory for eps_concentrated.
constexpr int kEpsHistLayers = 256;

// A layer as applied, kept on the host so that the waves that are not
// resident can be brought to the same point later; centre_sweep marks a
// measurement instead, whose centre moves (to site 0, then along the chain)
// the replay repeats so that every wave sees the same sequence of operations.
struct RecordedLayer {
  std::vector<int32_t> left_qubit;
  std::vector<double> gates, kraus;
  int32_t n_kraus = 0;
  double coin_p = 1.0;
  bool centre_sweep = false;
};

struct lemps_sim {
  lemps_config cfg;
  int n = 0;
  int64_t B = 0;             // trajectories of the resident wave (kernel grids, counts)
  int64_t Bcap = 0;          // wave capacity: allocation and per-trajectory strides
  int64_t n_total = 0;       // trajectories of the handle (all waves)
  int n_waves = 1;
  int wave = 0;              // the resident wave
  bool wave_current = true;  // the resident wave has every recorded layer applied
  int64_t wave_offset = 0;   // global id of the resident wave's first trajectory
  std::vector<RecordedLayer> history;   // every layer applied (multi-wave handles only)
  int chi = 0;
  int cap_max = 0;           // bond capacity: chi (local layering) or 2 chi (global)
  int prec = 0;
  cudaStream_t stream = nullptr;
  bool sticky = false;
  std::vector<std::pair<void*, size_t>> allocs;
  std::vector<int32_t> cap_h;
  std::vector<int64_t> off_h;
  size_t elem = 0;           // bytes per complex element of the MPS
  void* mps = nullptr;
  int64_t* site_off = nullptr;
  int32_t* cap = nullptr;
  int32_t* bond = nullptr;
  void* ws[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t ws_stride = 0;
  double* evals = nullptr;
  zd* rho12 = nullptr;
  zd* top = nullptr;
  double* eps_layer = nullptr;
  double* eps_tot = nullptr;
  double* disc_last = nullptr;
  int32_t* status = nullptr;
  int32_t* kept = nullptr;
  double* trace = nullptr;
  int8_t* blog = nullptr;
  int64_t log_cap = 0;
  zd* layer_buf = nullptr;   // gates + kraus of the current layer
  int64_t layer_cap = 0;     // complex numbers
  zd* haar = nullptr;        // Haar-optimal mode: [0, 4) rho = I/2, [4, 20) remixed set, [20] E_av
  zd* eye4 = nullptr;        // 4x4 identity: the gate of the noise and truncation passes
  double* eps_hist = nullptr;  // [B][kEpsHistLayers] per-layer 4 sqrt(2 sum eps)
  int layers_done = 0;
  uint8_t* bits_buf = nullptr;  // sample_bitstrings output (largest request so far)
  size_t bits_cap = 0;
  std::vector<double> haar_key;  // Kraus set (host) whose remix haar holds
  double* obs = nullptr;     // measure scratch: z [B][n], zz [B][n-1], s_half [B], eps_bound [B]
  double* stats = nullptr;   // reductions
  int64_t gates_done = 0;
  int center = 0;
  size_t mps_bytes = 0;
  // Tensor-core contraction (mixed precision): TMA maps of every site k with
  // cap[k], cap[k+1] >= 64, viewed as [2 cap[k]][cap[k+1]] complex64 rows over
  // all trajectories, with the A box (16 x 128) and the B box (cap[k+1] x 32).
  std::vector<CUtensorMap> map_a, map_b;
  std::vector<char> tc_site;
  // GEMM tile per kernel (0 contraction, 1 left Gram, 2 right Gram) and gate
  // position q: [3][n-1] indices into GemmTileShape, -1 where the tensor-core
  // contraction runs; chosen by the autotuner in sim_create (or fixed).
  std::vector<int8_t> tiles;
  double tune_ms = 0.0;
  int tile_of(int kind, int q) const { return tiles.empty() ? 0 : tiles[(size_t)kind * (n - 1) + q]; }
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;  // (kind, (start, stop))
  double prof_ms[LEMPS_NUM_KERNEL_KINDS] = {0};
  int64_t prof_n[LEMPS_NUM_KERNEL_KINDS] = {0};

  // Record an event pair around one launch when profiling.
  template <class F>
  void timed(int kind, F&& launch) {
    if (!profiling) { launch(); return; }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, stream);
    launch();
    cudaEventRecord(b, stream);
    prof.push_back({kind, {a, b}});
  }
  void collect_profile() {
    cudaStreamSynchronize(stream);
    for (auto& p : prof) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.second.first, p.second.second);
      prof_ms[p.first] += ms;
      prof_n[p.first] += 1;
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    prof.clear();
  }

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (cfg.alloc) {
      p = cfg.alloc(bytes, (void*)stream, cfg.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) allocs.push_back({p, bytes});
    return p;
  }
  void release() {
    for (auto& a : allocs) {
      if (cfg.free) cfg.free(a.first, a.second, (void*)stream, cfg.alloc_ctx);
      else cudaFree(a.first);
    }
    allocs.clear();
  }
  template <class R>
  SimView<R> view() const {
    SimView<R> v;
    v.mps = reinterpret_cast<cpx<R>*>(mps);
    v.site_off = site_off;
    v.cap = cap;
    v.bond = bond;
    v.n = n;
    v.B = B;
    v.chi = cap_max;   // evals stride (2 cap_max per trajectory)
    v.ws0 = reinterpret_cast<cpx<R>*>(ws[0]);
    v.ws1 = reinterpret_cast<cpx<R>*>(ws[1]);
    v.ws2 = reinterpret_cast<cpx<R>*>(ws[2]);
    v.ws3 = reinterpret_cast<cpx<R>*>(ws[3]);
    v.g64 = reinterpret_cast<zd*>(ws[1]);
    v.u64 = reinterpret_cast<zd*>(ws[2]);
    v.h64 = reinterpret_cast<zd*>(ws[3]);
    // complex128 eigenvectors in the FP64 mode, and in the mixed one on request
    v.u_fp64 = (sizeof(R) == 8 || cfg.eigvec_fp64) ? 1 : 0;
    v.ws_stride = ws_stride;
    v.evals = evals;
    v.rho12 = rho12;
    v.top = top;
    v.eps_layer = eps_layer;
    v.eps_tot = eps_tot;
    v.disc_last = disc_last;
    v.status = status;
    v.kept = kept;
    v.trace = trace;
    return v;
  }
};

namespace {

typedef CUresult (*TensorMapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
TensorMapEncodeFn tensor_map_encoder() {
  static TensorMapEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TensorMapEncodeFn>(p);
  }
  return fn;
}

// 3-D map over (column, row, trajectory) of the complex64 rows of one site:
// cols x rows per trajectory, 8-byte elements, trajectory stride cols * rows.
bool encode_site_map(CUtensorMap* m, void* base, int cols, int rows, int64_t ntraj, int box0, int box1,
                     CUtensorMapSwizzle swizzle) {
  TensorMapEncodeFn fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)ntraj};
  const cuuint64_t str[2] = {(cuuint64_t)cols * 8, (cuuint64_t)cols * 8 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, base, dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

lemps_status check_cuda(lemps_sim* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (h) h->sticky = true;
    return fail(LEMPS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  }
  return LEMPS_OK;
}

// Put wave w (global trajectory ids traj_offset + w Bcap onwards) in
// |0...0>, discarding the resident state; the wave then has no layer applied.
void reset_wave(lemps_sim* h, int w) {
  h->wave = w;
  h->wave_offset = h->cfg.traj_offset + (int64_t)w * h->Bcap;
  h->B = std::min<int64_t>(h->Bcap, h->n_total - (int64_t)w * h->Bcap);
  h->center = 0;
  h->gates_done = 0;
  h->layers_done = 0;
  h->wave_current = h->history.empty();
  cudaMemsetAsync(h->mps, 0, h->mps_bytes, h->stream);
  if (h->log_cap > 0) cudaMemsetAsync(h->blog, 0xff, h->log_cap * 2 * h->Bcap, h->stream);
  if (h->prec == LEMPS_FP64) k_init_state<double><<<(unsigned)h->B, 64, 0, h->stream>>>(h->view<double>());
  else k_init_state<float><<<(unsigned)h->B, 64, 0, h->stream>>>(h->view<float>());
}

// Centre moves and eigensolves whose matrices exceed the on-chip kernels
// (site capacities above 128) run the global-memory kernels of big_kernels.cuh.
bool big_move(const lemps_sim* h, int k) {
  return h->cfg.big_kernels || std::max(h->cap_h[k], h->cap_h[k + 1]) > 128;
}
bool big_gram(const lemps_sim* h, int q, int mode) {
  const int n = mode == 0 ? 2 * h->cap_h[q] : (mode == 1 ? 2 * h->cap_h[q + 2] : h->cap_h[q + 1]);
  return h->cfg.big_kernels || n > 256;
}

template <class R>
void launch_move(lemps_sim* h, int k, int dir) {
  if (big_move(h, k)) {
    h->timed(LEMPS_K_MOVE, [&] {
      k_move_center_big<R><<<(unsigned)h->B, kThreads, BigMoveSmem<R>::kBytes, h->stream>>>(h->view<R>(), k, dir);
    });
    return;
  }
  const size_t smem = sizeof(QrSmem<R>);
  static bool attr = false;  // one opt-in per instantiation
  if (!attr) {
    cudaFuncSetAttribute(k_move_center<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  h->timed(LEMPS_K_MOVE,
           [&] { k_move_center<R><<<(unsigned)h->B, kThreads, smem, h->stream>>>(h->view<R>(), k, dir); });
}

template <class R>
void move_center_to(lemps_sim* h, int target) {
  while (h->center < target) { launch_move<R>(h, h->center, +1); ++h->center; }
  while (h->center > target) { launch_move<R>(h, h->center, -1); --h->center; }
}

constexpr int kHeevThreads = 512;

// Hermitian eigensolve of the Gram matrix: tridiagonalization, eigenvalues and
// tridiagonal eigenvectors in complex128 in both precisions, the
// back-transformation (and U) in the storage precision;
// keeps the top min(chi_max, #{l > cutoff * trace}) eigenpairs (vectors = 1)
// or computes every eigenvalue (vectors = 0, cutoff = 0).
template <class RB>
void launch_heev_as(lemps_sim* h, const HeevView<double>& v, int q, int mode, double cutoff, int keep_max,
                    int vectors) {
  const size_t smem = HeevSmem<double>::kBytes;
  static bool attr = false;  // one opt-in per instantiation
  if (!attr) {
    cudaFuncSetAttribute(k_heev<double, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  h->timed(LEMPS_K_EIG, [&] {
    k_heev<double, RB><<<(unsigned)h->B, kHeevThreads, smem, h->stream>>>(v, q, mode, cutoff, keep_max, vectors);
  });
}

template <class RB>
void launch_heev_big(lemps_sim* h, const HeevView<double>& v, int q, int mode, double cutoff, int keep_max,
                     int vectors) {
  const size_t smem = sizeof(BigHeevSmem);
  static bool attr = false;  // one opt-in per instantiation
  if (!attr) {
    cudaFuncSetAttribute(k_heev_big<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  h->timed(LEMPS_K_EIG, [&] {
    k_heev_big<RB><<<(unsigned)h->B, kBigHeevThreads, smem, h->stream>>>(v, q, mode, cutoff, keep_max, vectors);
  });
}

template <class R>
void launch_heev(lemps_sim* h, int q, int mode, double cutoff, int keep_max, int vectors) {
  const SimView<R> sv = h->view<R>();
  if (big_gram(h, q, mode)) {
    if (sv.u_fp64) launch_heev_big<double>(h, heev_view(sv), q, mode, cutoff, keep_max, vectors);
    else launch_heev_big<float>(h, heev_view(sv), q, mode, cutoff, keep_max, vectors);
    return;
  }
  if (sv.u_fp64) launch_heev_as<double>(h, heev_view(sv), q, mode, cutoff, keep_max, vectors);
  else launch_heev_as<float>(h, heev_view(sv), q, mode, cutoff, keep_max, vectors);
}

// The SIMT contraction and the Gram kernel with the GEMM tile `tile`
// (an index into GemmTileShape<R, .>).
template <class R>
void contract_simt(const SimView<R>& sv, int q, int tile, cudaStream_t st) {
  const unsigned g = (unsigned)sv.B;
  switch (tile) {
    case 1: k_contract<R, 1><<<g, kThreads, 0, st>>>(sv, q); break;
    case 2: k_contract<R, 2><<<g, kThreads, 0, st>>>(sv, q); break;
    case 3: k_contract<R, 3><<<g, kThreads, 0, st>>>(sv, q); break;
    default: k_contract<R, 0><<<g, kThreads, 0, st>>>(sv, q);
  }
}

template <class R>
void apply_gram(const SimView<R>& sv, int q, int side, int tile, cudaStream_t st) {
  const unsigned g = (unsigned)sv.B;
  switch (tile) {
    case 1: k_apply_gram<R, 1><<<g, kThreads, 0, st>>>(sv, q, side); break;
    case 2: k_apply_gram<R, 2><<<g, kThreads, 0, st>>>(sv, q, side); break;
    case 3: k_apply_gram<R, 3><<<g, kThreads, 0, st>>>(sv, q, side); break;
    default: k_apply_gram<R, 0><<<g, kThreads, 0, st>>>(sv, q, side);
  }
}

void tile_shape(int prec, int id, int& bm, int& bn) {
  static const int f[kNumGemmTiles][2] = {{GemmTileShape<float, 0>::BM, GemmTileShape<float, 0>::BN},
                                          {GemmTileShape<float, 1>::BM, GemmTileShape<float, 1>::BN},
                                          {GemmTileShape<float, 2>::BM, GemmTileShape<float, 2>::BN},
                                          {GemmTileShape<float, 3>::BM, GemmTileShape<float, 3>::BN}};
  static const int d[kNumGemmTiles][2] = {{GemmTileShape<double, 0>::BM, GemmTileShape<double, 0>::BN},
                                          {GemmTileShape<double, 1>::BM, GemmTileShape<double, 1>::BN},
                                          {GemmTileShape<double, 2>::BM, GemmTileShape<double, 2>::BN},
                                          {GemmTileShape<double, 3>::BM, GemmTileShape<double, 3>::BN}};
  const int(*t)[2] = (prec == LEMPS_FP64) ? d : f;
  bm = t[id][0];
  bn = t[id][1];
}

// Tiles chosen so far in this process: (device, precision, kernel, full-SM
// batch, cap_q, cap_q+1, cap_q+2) -> tile index.
std::mutex g_tile_mu;
std::map<std::array<int, 7>, int> g_tile_record;

// GEMM tile autotuner, run by sim_create before the state is initialized.
// For each kernel (contraction, left Gram, right Gram) and each distinct
// triple of site capacities not yet in the process record, every candidate
// tile is timed on min(Bcap, 2 x #SMs) trajectories whose bonds are all at
// their capacities (operands zeroed; values do not change the timing): one
// warm-up launch, then three launches between CUDA events on the handle's
// stream.  The fastest is kept if it beats the default 64 x 64 by 3 %.
// Capacity triples above 128 keep the default: there one timing launch of a
// complex128 Gram product can take half a second.
// All candidates compute the same results bit for bit (each output entry is
// accumulated over k in order), so the choice only affects speed.
template <class R>
lemps_status autotune_tiles(lemps_sim* h) {
  const int n = h->n, np = n - 1;
  h->tiles.assign((size_t)3 * np, 0);
  h->tune_ms = 0.0;
  for (int q = 0; q < np; ++q)
    if (sizeof(R) == 4 && !h->tc_site.empty() && h->tc_site[q] && h->tc_site[q + 1]) h->tiles[q] = -1;
  if (h->cfg.gemm_tile > 0) {
    for (auto& t : h->tiles)
      if (t >= 0) t = (int8_t)(h->cfg.gemm_tile - 1);
    return LEMPS_OK;
  }
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return check_cuda(h, "sim_create: autotune device query");
  const int64_t Bt = std::min<int64_t>(h->Bcap, 2 * (int64_t)sms);
  auto key_of = [&](int kind, int q) {
    return std::array<int, 7>{dev, h->prec, kind, Bt >= sms ? 1 : 0, h->cap_h[q], h->cap_h[q + 1], h->cap_h[q + 2]};
  };
  auto tuned = [&](int q) { return std::max(h->cap_h[q], std::max(h->cap_h[q + 1], h->cap_h[q + 2])) <= 128; };
  std::vector<std::pair<int, int>> todo;   // (kind, first position) of each key still to time
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    std::map<std::array<int, 7>, int> seen;
    for (int kind = 0; kind < 3; ++kind)
      for (int q = 0; q < np; ++q) {
        if (h->tiles[(size_t)kind * np + q] < 0 || !tuned(q)) continue;
        const auto key = key_of(kind, q);
        if (g_tile_record.count(key) || seen.count(key)) continue;
        seen[key] = 1;
        todo.push_back({kind, q});
      }
  }
  if (!todo.empty()) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int32_t> bonds((size_t)Bt * (n + 1));
    for (int64_t t = 0; t < Bt; ++t)
      for (int k = 0; k <= n; ++k) bonds[(size_t)t * (n + 1) + k] = h->cap_h[k];
    cudaMemcpyAsync(h->bond, bonds.data(), sizeof(int32_t) * bonds.size(), cudaMemcpyHostToDevice, h->stream);
    cudaMemsetAsync(h->mps, 0, h->mps_bytes, h->stream);
    cudaMemsetAsync(h->ws[0], 0, h->elem * h->ws_stride * Bt, h->stream);
    cudaMemsetAsync(h->top, 0, sizeof(zd) * 16 * Bt, h->stream);
    SimView<R> v = h->view<R>();
    v.B = Bt;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<std::pair<std::array<int, 7>, int>> found;
    for (const auto& kq : todo) {
      const int kind = kq.first, q = kq.second;
      auto launch = [&](int tile) {
        if (kind == 0) contract_simt<R>(v, q, tile, h->stream);
        else apply_gram<R>(v, q, kind - 1, tile, h->stream);
      };
      float ms[kNumGemmTiles];
      for (int c = 0; c < kNumGemmTiles; ++c) {
        launch(c);
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < 3; ++r) launch(c);
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        ms[c] = 0.f;
        cudaEventElapsedTime(&ms[c], e0, e1);
      }
      int best = 0;
      for (int c = 1; c < kNumGemmTiles; ++c)
        if (ms[c] < ms[best]) best = c;
      if (!(ms[best] < 0.97f * ms[0])) best = 0;
      found.push_back({key_of(kind, q), best});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);   // the bond copy's host buffer
    lemps_status st = check_cuda(h, "sim_create: autotune");
    if (st != LEMPS_OK) return st;
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (const auto& f : found) g_tile_record.emplace(f.first, f.second);   // the first record of a key wins
    h->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  std::lock_guard<std::mutex> lk(g_tile_mu);
  for (int kind = 0; kind < 3; ++kind)
    for (int q = 0; q < np; ++q) {
      int8_t& t = h->tiles[(size_t)kind * np + q];
      if (t >= 0 && tuned(q)) t = (int8_t)g_tile_record.at(key_of(kind, q));
    }
  return LEMPS_OK;
}

// Two-site contraction of the pair (q, q+1): on the tensor cores in mixed
// precision when all three site capacities lie in [64, 128] (and are even),
// else the SIMT kernel with the handle's tile for q.
template <class R>
void launch_contract(lemps_sim* h, int q) {
  SimView<R> sv = h->view<R>();
  if (sizeof(R) == 4 && !h->tc_site.empty() && h->tc_site[q] && h->tc_site[q + 1]) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
      attr = true;
    }
    h->timed(LEMPS_K_CONTRACT, [&] {
      k_contract_tc<<<(unsigned)h->B, tc::kThreads, tc::kSmemBytes, h->stream>>>(
          h->map_a[q], h->map_b[q + 1], h->view<float>(), q);
    });
    return;
  }
  h->timed(LEMPS_K_CONTRACT, [&] { contract_simt<R>(sv, q, h->tile_of(0, q), h->stream); });
}

template <class R>
lemps_status apply_layer_t(lemps_sim* h, const lemps_layer* L) {
  const int ng = L->n_gates;
  const int64_t need = (int64_t)ng * 16 + (int64_t)L->n_kraus * 4;
  if (need > h->layer_cap) return fail(LEMPS_EINVAL, "apply_layer: too many gates for this handle");
  if (ng > 0) {
    if (cudaMemcpyAsync(h->layer_buf, L->gates, sizeof(zd) * 16 * ng, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return check_cuda(h, "apply_layer copy");
  }
  zd* kraus_d = h->layer_buf + 16 * (int64_t)ng;
  if (cudaMemcpyAsync(kraus_d, L->kraus, sizeof(zd) * 4 * L->n_kraus, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return check_cuda(h, "apply_layer copy");
  const zd* kset_d = kraus_d;
  int kset_r = L->n_kraus;
  int kmode = h->cfg.unravel_mode;
  if (kmode == LEMPS_UNRAVEL_HAAR_OPT) {
    // Remix the channel's Kraus set once for the Bell state (reduced state
    // I/2); every site then samples the remixed set as given.  The remix is
    // recomputed only when the layer's Kraus set changes.
    std::vector<double> key(L->kraus, L->kraus + 8 * L->n_kraus);
    if (key != h->haar_key) {
      h->timed(LEMPS_K_UNRAVEL, [&] {
        launch_unravel_batch(h->haar, kraus_d, L->n_kraus, 1, h->haar + 4, reinterpret_cast<double*>(h->haar + 20),
                             h->stream);
      });
      h->haar_key.swap(key);
    }
    kset_d = h->haar + 4;
    kset_r = 4;
    kmode = LEMPS_UNRAVEL_GIVEN;
  }
  const unsigned grid_t = (unsigned)((h->B + kThreads - 1) / kThreads);
  SimView<R> sv = h->view<R>();
  // One pair step: centre onto (q, q+1), contraction, gate and noise sites
  // (coin_p = 0: no noise, the gate alone), Gram on the given side,
  // eigensolve keeping at most keep_max, split.  gate_global keys the Philox
  // counters of the noise sites.
  auto pair_step = [&](int q, const zd* gate, int gate_local, double coin_p, int64_t gate_global, bool log,
                       int keep_max, int side) {
    if (h->center < q) move_center_to<R>(h, q);
    else if (h->center > q + 1) move_center_to<R>(h, q + 1);
    launch_contract<R>(h, q);
    LayerDev ld;
    ld.gates = gate;
    ld.kraus = kset_d;
    ld.r = kset_r;
    ld.coin_p = coin_p;
    ld.mode = kmode;
    ld.seed = h->cfg.seed;
    ld.traj_offset = h->wave_offset;
    ld.gate_global = gate_global;
    ld.gate_local = gate_local;
    ld.blog = (log && gate_global < h->log_cap) ? h->blog + gate_global * 2 * h->B : nullptr;
    GateState gs;
    gs.rho12 = h->rho12;
    gs.top = h->top;
    gs.status = h->status;
    gs.B = h->B;
    h->timed(LEMPS_K_UNRAVEL, [&] { launch_unravel_gate(gs, ld, h->stream); });
    h->timed(LEMPS_K_GRAM, [&] { apply_gram<R>(sv, q, side, h->tile_of(1 + side, q), h->stream); });
    launch_heev<R>(h, q, side, h->cfg.trunc_cutoff, keep_max, 1);
    h->timed(LEMPS_K_SPLIT, [&] { k_split<R><<<(unsigned)h->B, kThreads, 0, h->stream>>>(sv, q, side); });
    h->center = (side == 0) ? q + 1 : q;
  };
  // side 0 (centre to q+1) when the next pair lies to the right
  auto side_of = [&](int g) {
    const int q = L->left_qubit[g];
    if (g + 1 < ng) return (L->left_qubit[g + 1] > q) ? 0 : 1;
    if (g > 0) return (q > L->left_qubit[g - 1]) ? 0 : 1;
    return 0;
  };
  // Gram side of a gate's split in the local layering: the smaller Gram matrix
  // when the site capacities around the pair differ (the eigensolve costs ~
  // size^3, and a centre left one site away from the next pair costs one more
  // QR move, far less), else the side that leaves the centre next to the
  // following pair.  Both sides give the same truncated split (Sec. IV.A's
  // SVD re-split seen from either side), up to rounding.
  auto split_side = [&](int g) {
    const int q = L->left_qubit[g];
    const int cl = h->cap_h[q], cr = h->cap_h[q + 2];
    if (cl != cr) return cl < cr ? 0 : 1;
    return side_of(g);
  };
  if (h->cfg.layering == LEMPS_LAYER_GLOBAL) {
    // all gates (no noise, bonds up to 2 chi), then the noise on every gated
    // pair with the identity gate and the same Philox counters as the local
    // layering, then a left-to-right truncation sweep over every bond
    for (int g = 0; g < ng; ++g)
      pair_step(L->left_qubit[g], h->layer_buf + 16 * (int64_t)g, 0, 0.0, h->gates_done + g, false, h->cap_max,
                side_of(g));
    for (int g = 0; g < ng; ++g)
      pair_step(L->left_qubit[g], h->eye4, 0, L->coin_p, h->gates_done + g, true, h->cap_max, side_of(g));
    for (int k = 0; k + 1 < h->n; ++k) pair_step(k, h->eye4, 0, 0.0, h->gates_done, false, h->chi, 0);
  } else {
    for (int g = 0; g < ng; ++g)
      pair_step(L->left_qubit[g], h->layer_buf, g, L->coin_p, h->gates_done + g, true, h->chi, split_side(g));
  }
  double* hist = (h->layers_done < kEpsHistLayers) ? h->eps_hist : nullptr;
  h->timed(LEMPS_K_OTHER, [&] {
    k_layer_end<R><<<grid_t, kThreads, 0, h->stream>>>(sv, hist, kEpsHistLayers, h->layers_done);
  });
  ++h->layers_done;
  h->gates_done += ng;
  return check_cuda(h, "apply_layer");
}

__global__ void k_finalize_obs(const double* eps_tot, double eps_max, int64_t B, double* eps_bound) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B) return;
  double e = eps_tot[t];
  eps_bound[t] = (e <= eps_max - 2.0) ? e : eps_max;
}

// mean and standard error of column c of a [B][ncol] array (one block per column)
__global__ void k_column_stats(const double* x, int64_t B, int ncol, double* mean, double* se) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < B; t += blockDim.x) s += x[t * ncol + c];
  s = block_sum(s, red);
  const double m = s / (double)B;
  double v = 0.0;
  for (int64_t t = threadIdx.x; t < B; t += blockDim.x) {
    double d = x[t * ncol + c] - m;
    v += d * d;
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    mean[c] = m;
    se[c] = B > 1 ? sqrt(v / (double)(B - 1) / (double)B) : 0.0;
  }
}

template <class R>
lemps_status measure_t(lemps_sim* h, lemps_measurement* m) {
  const int n = h->n;
  const int64_t B = h->B;
  const unsigned grid_t = (unsigned)((B + kThreads - 1) / kThreads);
  SimView<R> sv = h->view<R>();
  double* z = h->obs;
  double* zz = z + B * n;
  double* sh = zz + B * (n - 1);
  double* eb = sh + B;
  move_center_to<R>(h, 0);
  const int hb = n / 2;  // bond n/2 lies between sites hb-1 and hb
  for (int q = 0; q + 1 < n; ++q) {
    launch_contract<R>(h, q);
    k_obs_from_rho12<<<grid_t, kThreads, 0, h->stream>>>(h->rho12, B, n, q, z, zz);
    if (q == hb - 1) {
      k_site_gram<R><<<(unsigned)B, kThreads, 0, h->stream>>>(sv, q);
      launch_heev<R>(h, q, 2, 0.0, h->cap_max, 0);
      k_entropy_from_evals<<<grid_t, kThreads, 0, h->stream>>>(h->evals, 2 * h->cap_max, h->bond, n + 1, q + 1, B, sh);
    }
    launch_move<R>(h, q, +1);
    ++h->center;
  }
  k_finalize_obs<<<grid_t, kThreads, 0, h->stream>>>(h->eps_tot, h->cfg.eps_max, B, eb);
  double* st = h->stats;  // z_mean n, z_se n, zz_mean n-1, zz_se n-1, sh 2, eb 2
  k_column_stats<<<n, kThreads, 0, h->stream>>>(z, B, n, st, st + n);
  k_column_stats<<<n - 1, kThreads, 0, h->stream>>>(zz, B, n - 1, st + 2 * n, st + 3 * n - 1);
  k_column_stats<<<1, kThreads, 0, h->stream>>>(sh, B, 1, st + 4 * n - 2, st + 4 * n - 1);
  k_column_stats<<<1, kThreads, 0, h->stream>>>(eb, B, 1, st + 4 * n, st + 4 * n + 1);
  lemps_status cs = check_cuda(h, "measure");
  if (cs != LEMPS_OK) return cs;
  std::vector<double> hs(4 * n + 2);
  std::vector<int32_t> stat(B);
  if (cudaMemcpyAsync(hs.data(), st, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(stat.data(), h->status, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return check_cuda(h, "measure copy");
  if (m->z) cudaMemcpyAsync(m->z, z, sizeof(double) * B * n, cudaMemcpyDeviceToHost, h->stream);
  if (m->zz) cudaMemcpyAsync(m->zz, zz, sizeof(double) * B * (n - 1), cudaMemcpyDeviceToHost, h->stream);
  if (m->s_half) cudaMemcpyAsync(m->s_half, sh, sizeof(double) * B, cudaMemcpyDeviceToHost, h->stream);
  if (m->eps_bound) cudaMemcpyAsync(m->eps_bound, eb, sizeof(double) * B, cudaMemcpyDeviceToHost, h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "measure sync");
  if (m->status) std::memcpy(m->status, stat.data(), sizeof(int32_t) * B);
  for (int i = 0; i < n; ++i) { m->z_mean[i] = hs[i]; m->z_stderr[i] = hs[n + i]; }
  for (int i = 0; i + 1 < n; ++i) { m->zz_mean[i] = hs[2 * n + i]; m->zz_stderr[i] = hs[3 * n - 1 + i]; }
  m->s_half_mean = hs[4 * n - 2];
  m->s_half_stderr = hs[4 * n - 1];
  m->eps_hat = hs[4 * n];
  m->eps_buffer = std::sqrt(h->cfg.eps_max * h->cfg.eps_max / (2.0 * (double)B) * std::log(1.0 / 0.05));
  int64_t nf = 0;
  for (int64_t t = 0; t < B; ++t) nf += (stat[t] != 0);
  m->n_failed = nf;
  return nf ? fail(LEMPS_ENUMERIC, "measure: some trajectories flagged a numerical failure") : LEMPS_OK;
}

}  // namespace

extern "C" {

const char* lemps_last_error(void) { return g_err.c_str(); }

// Shared with the other translation units of the library (not in lemps.h).
lemps_status lemps_set_error_(int st, const char* msg) {
  g_err = msg;
  return (lemps_status)st;
}

lemps_status sim_create(const lemps_config* cfg, lemps_handle* out) {
  if (!cfg || !out) return fail(LEMPS_EINVAL, "sim_create: null argument");
  *out = nullptr;
  if (cfg->n_qubits < 2 || cfg->n_qubits > 4096) return fail(LEMPS_EINVAL, "sim_create: n_qubits out of range");
  if (cfg->chi_max < 1 || cfg->chi_max > 512) return fail(LEMPS_EINVAL, "sim_create: chi_max must be in 1..512");
  if (cfg->n_traj < 1) return fail(LEMPS_EINVAL, "sim_create: n_traj must be positive");
  if (cfg->precision != LEMPS_FP64 && cfg->precision != LEMPS_MIXED) return fail(LEMPS_EINVAL, "sim_create: bad precision");
  if (cfg->unravel_mode != LEMPS_UNRAVEL_OPTIMAL && cfg->unravel_mode != LEMPS_UNRAVEL_GIVEN &&
      cfg->unravel_mode != LEMPS_UNRAVEL_HAAR_OPT)
    return fail(LEMPS_EINVAL, "sim_create: bad unravel_mode");
  if (!(cfg->trunc_cutoff >= 0.0) || !(cfg->eps_max >= 2.0)) return fail(LEMPS_EINVAL, "sim_create: bad cutoff or eps_max");
  if (cfg->layering != LEMPS_LAYER_LOCAL && cfg->layering != LEMPS_LAYER_GLOBAL)
    return fail(LEMPS_EINVAL, "sim_create: bad layering");
  if (cfg->layering == LEMPS_LAYER_GLOBAL && cfg->chi_max > 64)
    return fail(LEMPS_EINVAL, "sim_create: global layering holds bonds of 2 chi_max, so chi_max must be <= 64");
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return fail(LEMPS_EINVAL, "sim_create: alloc and free go together");
  if (cfg->max_traj_in_flight < 0) return fail(LEMPS_EINVAL, "sim_create: max_traj_in_flight must be >= 0");
  if (cfg->eigvec_fp64 != 0 && cfg->eigvec_fp64 != 1) return fail(LEMPS_EINVAL, "sim_create: eigvec_fp64 must be 0 or 1");
  if (cfg->big_kernels != 0 && cfg->big_kernels != 1) return fail(LEMPS_EINVAL, "sim_create: big_kernels must be 0 or 1");
  if (cfg->gemm_tile < 0 || cfg->gemm_tile > kNumGemmTiles)
    return fail(LEMPS_EINVAL, "sim_create: gemm_tile must be 0 (autotune) or 1..4");
  lemps_sim* h = new lemps_sim();
  h->cfg = *cfg;
  h->n = cfg->n_qubits;
  h->n_total = cfg->n_traj;
  h->chi = cfg->chi_max;
  h->cap_max = (cfg->layering == LEMPS_LAYER_GLOBAL) ? 2 * cfg->chi_max : cfg->chi_max;
  h->prec = cfg->precision;
  h->stream = (cudaStream_t)cfg->cuda_stream;
  h->elem = (h->prec == LEMPS_FP64) ? sizeof(zd) : sizeof(zf);
  const int n = h->n;
  h->cap_h.resize(n + 1);
  for (int k = 0; k <= n; ++k) {
    int e = std::min(k, n - k);
    int64_t c = (e >= 30) ? (int64_t)1 << 30 : ((int64_t)1 << e);
    h->cap_h[k] = (int32_t)std::min<int64_t>(c, h->cap_max);
  }
  h->ws_stride = (int64_t)(2 * h->cap_max) * (2 * h->cap_max);
  h->log_cap = cfg->log_capacity > 0 ? cfg->log_capacity : 0;
  // Waves: the device holds Bcap trajectories at a time.  Bytes per
  // trajectory: the MPS slots, the four workspaces (the last three in
  // complex128), and the per-trajectory scalars and logs.
  {
    int64_t slot = 0;
    for (int k = 0; k < n; ++k) slot += (int64_t)h->cap_h[k] * 2 * h->cap_h[k + 1];
    const double per = (double)h->elem * (double)slot + (double)(h->elem + 3 * sizeof(zd)) * (double)h->ws_stride +
                       8.0 * (2 * h->cap_max + 2 * n + 1 + kEpsHistLayers + 8) + 4.0 * (n + 4) + 32.0 * 16 +
                       2.0 * (double)h->log_cap;
    int64_t cap = cfg->max_traj_in_flight;
    if (cap == 0) {
      // automatic: at most 60 % of the device's memory, and of what is free
      size_t fr = 0, totm = 0;
      if (cudaMemGetInfo(&fr, &totm) != cudaSuccess) {
        delete h;
        return fail(LEMPS_ECUDA, "sim_create: cudaMemGetInfo failed");
      }
      const double budget = std::min(0.6 * (double)totm, 0.9 * (double)fr);
      cap = std::max<int64_t>(1, (int64_t)(budget / per));
    }
    h->Bcap = std::min<int64_t>(cap, h->n_total);
    h->n_waves = (int)((h->n_total + h->Bcap - 1) / h->Bcap);
    h->B = h->Bcap;
  }
  h->off_h.resize(n);
  int64_t tot = 0;
  for (int k = 0; k < n; ++k) {
    h->off_h[k] = tot;
    tot += (int64_t)h->cap_h[k] * 2 * h->cap_h[k + 1] * h->Bcap;
  }
  h->layer_cap = (int64_t)(n / 2 + 1) * 16 + 4 * kMaxKraus;
  bool ok = true, aligned = true;
  auto A = [&](size_t bytes) {
    void* p = h->dalloc(bytes);
    if (!p) ok = false;
    if (((uintptr_t)p & 15) != 0) aligned = false;
    return p;
  };
  h->mps = A(h->elem * tot);
  h->site_off = (int64_t*)A(sizeof(int64_t) * n);
  h->cap = (int32_t*)A(sizeof(int32_t) * (n + 1));
  h->bond = (int32_t*)A(sizeof(int32_t) * (n + 1) * h->Bcap);
  // ws0 (two-site tensor) in the storage precision; ws1..ws3 at 16 bytes per
  // entry: the Gram matrix, eigenvectors and reflectors are complex128
  h->ws[0] = A(h->elem * h->ws_stride * h->Bcap);
  for (int i = 1; i < 4; ++i) h->ws[i] = A(sizeof(zd) * h->ws_stride * h->Bcap);
  h->evals = (double*)A(sizeof(double) * 2 * h->cap_max * h->Bcap);
  h->rho12 = (zd*)A(sizeof(zd) * 16 * h->Bcap);
  h->top = (zd*)A(sizeof(zd) * 16 * h->Bcap);
  h->eps_layer = (double*)A(sizeof(double) * h->Bcap);
  h->eps_tot = (double*)A(sizeof(double) * h->Bcap);
  h->disc_last = (double*)A(sizeof(double) * h->Bcap);
  h->status = (int32_t*)A(sizeof(int32_t) * h->Bcap);
  h->kept = (int32_t*)A(sizeof(int32_t) * h->Bcap);
  h->trace = (double*)A(sizeof(double) * h->Bcap);
  h->blog = (int8_t*)A(std::max<int64_t>(1, h->log_cap * 2 * h->Bcap));
  h->layer_buf = (zd*)A(sizeof(zd) * h->layer_cap);
  h->haar = (zd*)A(sizeof(zd) * 21);
  h->eye4 = (zd*)A(sizeof(zd) * 16);
  h->eps_hist = (double*)A(sizeof(double) * kEpsHistLayers * h->Bcap);
  h->obs = (double*)A(sizeof(double) * h->Bcap * (2 * n + 1));
  h->stats = (double*)A(sizeof(double) * (4 * n + 4));
  if (!ok || !aligned) {
    h->release();
    delete h;
    return ok ? fail(LEMPS_EINVAL, "sim_create: the allocator returned a block that is not 16-byte aligned")
              : fail(LEMPS_ENOMEM, "sim_create: device allocation failed");
  }
  h->mps_bytes = h->elem * tot;
  if (h->prec == LEMPS_MIXED) {
    // tensor maps of the sites the tensor-core contraction can take: site k
    // as the left operand (box of 8 complex columns x 128 rows, 64-byte
    // swizzle: two M tiles cover 2 cap_k <= 256 rows) and as the right
    // operand (box of all cap_{k+1} <= 128 columns x 16 rows 2k' + s)
    h->map_a.resize(n);
    h->map_b.resize(n);
    h->tc_site.assign(n, 0);
    for (int k = 0; k < n; ++k) {
      const int rows = 2 * h->cap_h[k], cols = h->cap_h[k + 1];
      if (h->cap_h[k] < 64 || h->cap_h[k] > 128 || cols < 64 || cols > 128 || cols % 2) continue;
      void* base = (char*)h->mps + h->off_h[k] * h->elem;
      if (!encode_site_map(&h->map_a[k], base, cols, rows, h->Bcap, tc::kKC, 128, CU_TENSOR_MAP_SWIZZLE_64B) ||
          !encode_site_map(&h->map_b[k], base, cols, rows, h->Bcap, cols, 2 * tc::kKC, CU_TENSOR_MAP_SWIZZLE_NONE)) {
        h->release();
        delete h;
        return fail(LEMPS_ECUDA, "sim_create: cuTensorMapEncodeTiled is unavailable or refused a site map");
      }
      h->tc_site[k] = 1;
    }
  }
  cudaMemcpyAsync(h->site_off, h->off_h.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->cap, h->cap_h.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, h->stream);
  {
    // the Bell state's reduced state, input of the Haar-optimal remix
    static const zd kHalfIdentity[4] = {{0.5, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.5, 0.0}};
    cudaMemcpyAsync(h->haar, kHalfIdentity, sizeof(kHalfIdentity), cudaMemcpyHostToDevice, h->stream);
    static const zd kEye4[16] = {{1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0},
                                 {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}};
    cudaMemcpyAsync(h->eye4, kEye4, sizeof(kEye4), cudaMemcpyHostToDevice, h->stream);
  }
  {
    lemps_status ts = (h->prec == LEMPS_FP64) ? autotune_tiles<double>(h) : autotune_tiles<float>(h);
    if (ts != LEMPS_OK) {
      cudaStreamSynchronize(h->stream);
      h->release();
      delete h;
      return ts;
    }
  }
  reset_wave(h, 0);
  lemps_status st = check_cuda(h, "sim_create");
  if (st != LEMPS_OK) {
    h->release();
    delete h;
    return st;
  }
  // The host vectors passed to cudaMemcpyAsync must outlive the copies.
  cudaStreamSynchronize(h->stream);
  *out = h;
  return LEMPS_OK;
}

lemps_status apply_layer(lemps_handle h, const lemps_layer* layer) {
  if (!h || !layer) return fail(LEMPS_EINVAL, "apply_layer: null argument");
  if (h->sticky) return fail(LEMPS_ECUDA, "apply_layer: handle has a sticky CUDA error");
  if (layer->n_gates < 0 || (layer->n_gates > 0 && (!layer->left_qubit || !layer->gates)) || !layer->kraus)
    return fail(LEMPS_EINVAL, "apply_layer: bad layer arrays");
  const int max_kraus = (h->cfg.unravel_mode == LEMPS_UNRAVEL_GIVEN) ? kMaxKraus : 4;
  if (layer->n_kraus < 1 || layer->n_kraus > max_kraus)
    return fail(LEMPS_EINVAL, "apply_layer: n_kraus must be 1..4 (1..8 in the given mode)");
  if (!(layer->coin_p >= 0.0 && layer->coin_p <= 1.0)) return fail(LEMPS_EINVAL, "apply_layer: coin_p outside [0,1]");
  std::vector<char> used(h->n, 0);
  for (int g = 0; g < layer->n_gates; ++g) {
    int q = layer->left_qubit[g];
    if (q < 0 || q + 1 >= h->n) return fail(LEMPS_EINVAL, "apply_layer: gate qubit out of range");
    if (used[q] || used[q + 1]) return fail(LEMPS_EINVAL, "apply_layer: gates of a layer must act on disjoint pairs");
    used[q] = used[q + 1] = 1;
  }
  for (int i = 0; i < layer->n_gates * 32; ++i)
    if (!std::isfinite(layer->gates[i])) return fail(LEMPS_EINVAL, "apply_layer: non-finite gate entry");
  // sum K^dagger K = I
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < layer->n_kraus; ++k) {
    const double* K = layer->kraus + 8 * k;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l < 2; ++l) {
          double ar = K[(l * 2 + i) * 2], ai = -K[(l * 2 + i) * 2 + 1];
          double br = K[(l * 2 + j) * 2], bi = K[(l * 2 + j) * 2 + 1];
          s[(i * 2 + j) * 2] += ar * br - ai * bi;
          s[(i * 2 + j) * 2 + 1] += ar * bi + ai * br;
        }
  }
  double dev = std::fabs(s[0] - 1) + std::fabs(s[6] - 1) + std::fabs(s[1]) + std::fabs(s[7]) + std::fabs(s[2]) +
               std::fabs(s[3]) + std::fabs(s[4]) + std::fabs(s[5]);
  if (!(dev < 1e-9)) return fail(LEMPS_EINVAL, "apply_layer: Kraus set is not trace preserving");
  if (h->n_waves > 1) {
    // kept for the waves that are not resident (replayed by measure)
    RecordedLayer r;
    r.left_qubit.assign(layer->left_qubit, layer->left_qubit + layer->n_gates);
    r.gates.assign(layer->gates, layer->gates + 32 * (size_t)layer->n_gates);
    r.kraus.assign(layer->kraus, layer->kraus + 8 * (size_t)layer->n_kraus);
    r.n_kraus = layer->n_kraus;
    r.coin_p = layer->coin_p;
    h->history.push_back(std::move(r));
  }
  if (h->prec == LEMPS_FP64) return apply_layer_t<double>(h, layer);
  return apply_layer_t<float>(h, layer);
}

lemps_status unravel_opt(const double* rho_a, const double* kraus, int32_t n_kraus, int64_t batch, double* kraus_out,
                         double* e_av, void* stream) {
  if (!rho_a || !kraus || !kraus_out || batch < 0) return fail(LEMPS_EINVAL, "unravel_opt: bad argument");
  if (n_kraus < 1 || n_kraus > 4) return fail(LEMPS_EINVAL, "unravel_opt: n_kraus must be 1..4");
  if (batch == 0) return LEMPS_OK;
  launch_unravel_batch((const zd*)rho_a, (const zd*)kraus, n_kraus, batch, (zd*)kraus_out, e_av, (cudaStream_t)stream);
  return check_cuda(nullptr, "unravel_opt");
}

lemps_status sample_branch(lemps_handle h, int64_t gate, int32_t slot, int32_t* branch_out) {
  if (!h || !branch_out || slot < 0 || slot > 1) return fail(LEMPS_EINVAL, "sample_branch: bad argument");
  if (h->n_waves > 1) return fail(LEMPS_ESTATE, "sample_branch: the handle runs in waves; per-trajectory inspection needs n_traj <= max_traj_in_flight");
  if (h->sticky) return fail(LEMPS_ECUDA, "sample_branch: sticky CUDA error");
  if (gate < 0 || gate >= h->gates_done) return fail(LEMPS_ESTATE, "sample_branch: gate not applied yet");
  if (gate >= h->log_cap) return fail(LEMPS_ESTATE, "sample_branch: gate beyond log_capacity");
  std::vector<int8_t> tmp(h->B);
  if (cudaMemcpyAsync(tmp.data(), h->blog + (gate * 2 + slot) * h->B, h->B, cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return check_cuda(h, "sample_branch");
  for (int64_t t = 0; t < h->B; ++t) branch_out[t] = tmp[t];
  return LEMPS_OK;
}

lemps_status sample_bitstrings(lemps_handle h, int32_t n_shots, uint8_t* bits_out) {
  if (!h || !bits_out || n_shots < 1 || n_shots > 65535) return fail(LEMPS_EINVAL, "sample_bitstrings: bad argument");
  if (h->n_waves > 1) return fail(LEMPS_ESTATE, "sample_bitstrings: the handle runs in waves; per-trajectory inspection needs n_traj <= max_traj_in_flight");
  if (h->sticky) return fail(LEMPS_ECUDA, "sample_bitstrings: sticky CUDA error");
  if (h->cap_max > 256) return fail(LEMPS_EINVAL, "sample_bitstrings: bond dimensions above 256 are not supported");
  const size_t bytes = (size_t)h->B * (size_t)n_shots * (size_t)h->n;
  if (bytes > h->bits_cap) {
    uint8_t* p = (uint8_t*)h->dalloc(bytes);
    if (!p) return fail(LEMPS_ENOMEM, "sample_bitstrings: device allocation failed");
    h->bits_buf = p;
    h->bits_cap = bytes;
  }
  const dim3 grid((unsigned)h->B, (unsigned)n_shots);
  if (h->prec == LEMPS_FP64) {
    move_center_to<double>(h, 0);
    k_sample_bits<double><<<grid, 256, 0, h->stream>>>(h->view<double>(), n_shots, h->cfg.seed, h->cfg.traj_offset,
                                                      h->bits_buf);
  } else {
    move_center_to<float>(h, 0);
    k_sample_bits<float><<<grid, 256, 0, h->stream>>>(h->view<float>(), n_shots, h->cfg.seed, h->cfg.traj_offset,
                                                     h->bits_buf);
  }
  if (cudaMemcpyAsync(bits_out, h->bits_buf, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return check_cuda(h, "sample_bitstrings copy");
  cudaStreamSynchronize(h->stream);
  return check_cuda(h, "sample_bitstrings");
}

lemps_status eps_concentrated(lemps_handle h, int32_t kind, double param, double* eps_out, double* eps_hat) {
  if (!h || !eps_hat) return fail(LEMPS_EINVAL, "eps_concentrated: null argument");
  if (h->n_waves > 1) return fail(LEMPS_ESTATE, "eps_concentrated: the handle runs in waves; per-trajectory inspection needs n_traj <= max_traj_in_flight");
  if (h->sticky) return fail(LEMPS_ECUDA, "eps_concentrated: sticky CUDA error");
  if (kind == 0 ? !(param > 0.0 && param <= 1.0) : (kind == 1 ? !(param >= 0.0 && param <= 1.0) : true))
    return fail(LEMPS_EINVAL, "eps_concentrated: kind 0 needs 0 < alpha <= 1, kind 1 needs 0 <= p <= 1");
  if (h->layers_done > kEpsHistLayers)
    return fail(LEMPS_ESTATE, "eps_concentrated: more than 256 layers since sim_create (history is full)");
  double* out = h->obs;   // measure scratch, [B] at least
  const unsigned grid_t = (unsigned)((h->B + kThreads - 1) / kThreads);
  k_eps_weighted<<<grid_t, kThreads, 0, h->stream>>>(h->eps_hist, kEpsHistLayers, h->B, h->layers_done, kind, param,
                                                     h->n, h->cfg.eps_max, out);
  std::vector<double> host((size_t)h->B);
  if (cudaMemcpyAsync(host.data(), out, sizeof(double) * h->B, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return check_cuda(h, "eps_concentrated copy");
  cudaStreamSynchronize(h->stream);
  lemps_status st = check_cuda(h, "eps_concentrated");
  if (st != LEMPS_OK) return st;
  double sum = 0.0;
  for (double x : host) sum += x;
  *eps_hat = sum / (double)h->B;
  if (eps_out) std::memcpy(eps_out, host.data(), sizeof(double) * h->B);
  return LEMPS_OK;
}

lemps_status measure(lemps_handle h, lemps_measurement* m) {
  if (!h || !m || !m->z_mean || !m->z_stderr || !m->zz_mean || !m->zz_stderr) return fail(LEMPS_EINVAL, "measure: bad argument");
  if (h->sticky) return fail(LEMPS_ECUDA, "measure: sticky CUDA error");
  auto measure_resident = [&](lemps_measurement* mw) {
    return (h->prec == LEMPS_FP64) ? measure_t<double>(h, mw) : measure_t<float>(h, mw);
  };
  if (h->n_waves == 1) return measure_resident(m);
  // Waves: the resident wave is measured as it stands, every other wave is
  // put in |0...0> and brought through the recorded layers first.  The
  // per-wave means and standard errors are merged exactly (sums of squared
  // deviations combined pairwise); the last wave processed stays resident.
  const int n = h->n;
  const int ncol = 2 * n + 1;   // z (n), zz (n - 1), s_half (1), eps_bound (1)
  std::vector<double> mean(ncol, 0.0), m2(ncol, 0.0);
  int64_t count = 0, failed = 0;
  std::vector<int> order;
  order.push_back(h->wave);
  for (int w = 0; w < h->n_waves; ++w)
    if (w != h->wave) order.push_back(w);
  for (int w : order) {
    if (w != h->wave || !h->wave_current) {
      reset_wave(h, w);
      for (const RecordedLayer& r : h->history) {
        if (r.centre_sweep) {
          if (h->prec == LEMPS_FP64) { move_center_to<double>(h, 0); move_center_to<double>(h, h->n - 1); }
          else { move_center_to<float>(h, 0); move_center_to<float>(h, h->n - 1); }
          continue;
        }
        lemps_layer L;
        L.n_gates = (int32_t)r.left_qubit.size();
        L.left_qubit = r.left_qubit.data();
        L.gates = r.gates.data();
        L.n_kraus = r.n_kraus;
        L.kraus = r.kraus.data();
        L.coin_p = r.coin_p;
        const lemps_status st = (h->prec == LEMPS_FP64) ? apply_layer_t<double>(h, &L) : apply_layer_t<float>(h, &L);
        if (st != LEMPS_OK) return st;
      }
      h->wave_current = true;
    }
    const int64_t off = (int64_t)w * h->Bcap, bw = h->B;
    std::vector<double> zm(n), zs(n), zzm(n > 1 ? n - 1 : 1), zzs(n > 1 ? n - 1 : 1);
    lemps_measurement mw{};
    mw.z = m->z ? m->z + off * n : nullptr;
    mw.zz = m->zz ? m->zz + off * (n - 1) : nullptr;
    mw.s_half = m->s_half ? m->s_half + off : nullptr;
    mw.eps_bound = m->eps_bound ? m->eps_bound + off : nullptr;
    mw.status = m->status ? m->status + off : nullptr;
    mw.z_mean = zm.data();
    mw.z_stderr = zs.data();
    mw.zz_mean = zzm.data();
    mw.zz_stderr = zzs.data();
    const lemps_status st = measure_resident(&mw);
    if (st != LEMPS_OK && st != LEMPS_ENUMERIC) return st;
    failed += mw.n_failed;
    // the wave's column statistics: mean and M2 = se^2 (B - 1) B
    std::vector<double> wm(ncol), ws(ncol);
    for (int i = 0; i < n; ++i) { wm[i] = zm[i]; ws[i] = zs[i]; }
    for (int i = 0; i + 1 < n; ++i) { wm[n + i] = zzm[i]; ws[n + i] = zzs[i]; }
    wm[2 * n - 1] = mw.s_half_mean; ws[2 * n - 1] = mw.s_half_stderr;
    wm[2 * n] = mw.eps_hat; ws[2 * n] = 0.0;
    for (int c = 0; c < ncol; ++c) {
      const double m2w = ws[c] * ws[c] * (double)(bw - 1) * (double)bw;
      if (count == 0) {
        mean[c] = wm[c];
        m2[c] = m2w;
      } else {
        const double tot = (double)(count + bw), d = wm[c] - mean[c];
        mean[c] += d * (double)bw / tot;
        m2[c] += m2w + d * d * (double)count * (double)bw / tot;
      }
    }
    count += bw;
  }
  {
    RecordedLayer sweep;
    sweep.centre_sweep = true;
    h->history.push_back(std::move(sweep));
  }
  auto se = [&](int c) { return count > 1 ? std::sqrt(m2[c] / (double)(count - 1) / (double)count) : 0.0; };
  for (int i = 0; i < n; ++i) { m->z_mean[i] = mean[i]; m->z_stderr[i] = se(i); }
  for (int i = 0; i + 1 < n; ++i) { m->zz_mean[i] = mean[n + i]; m->zz_stderr[i] = se(n + i); }
  m->s_half_mean = mean[2 * n - 1];
  m->s_half_stderr = se(2 * n - 1);
  m->eps_hat = mean[2 * n];
  m->eps_buffer = std::sqrt(h->cfg.eps_max * h->cfg.eps_max / (2.0 * (double)count) * std::log(1.0 / 0.05));
  m->n_failed = failed;
  return failed ? fail(LEMPS_ENUMERIC, "measure: some trajectories flagged a numerical failure") : LEMPS_OK;
}

lemps_status sim_waves(lemps_handle h, int64_t* wave_size, int32_t* n_waves) {
  if (!h || !wave_size || !n_waves) return fail(LEMPS_EINVAL, "sim_waves: null argument");
  *wave_size = h->Bcap;
  *n_waves = h->n_waves;
  return LEMPS_OK;
}

lemps_status sim_export_mps(lemps_handle h, int64_t traj, int32_t* bond_dims, double* tensors) {
  if (!h || !bond_dims || !tensors || traj < 0 || traj >= h->B) return fail(LEMPS_EINVAL, "sim_export_mps: bad argument");
  if (h->n_waves > 1) return fail(LEMPS_ESTATE, "sim_export_mps: the handle runs in waves; per-trajectory inspection needs n_traj <= max_traj_in_flight");
  if (h->sticky) return fail(LEMPS_ECUDA, "sim_export_mps: sticky CUDA error");
  const int n = h->n;
  if (cudaMemcpyAsync(bond_dims, h->bond + traj * (n + 1), sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return check_cuda(h, "sim_export_mps");
  int64_t out = 0;
  for (int k = 0; k < n; ++k) {
    const int cl = h->cap_h[k], cr = h->cap_h[k + 1];
    const int64_t slot = (int64_t)cl * 2 * cr;
    std::vector<char> buf(slot * h->elem);
    const char* src = (const char*)h->mps + (h->off_h[k] + traj * slot) * h->elem;
    if (cudaMemcpy(buf.data(), src, buf.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return check_cuda(h, "sim_export_mps");
    const int dl = bond_dims[k], dr = bond_dims[k + 1];
    for (int r = 0; r < 2 * dl; ++r)
      for (int b = 0; b < dr; ++b) {
        const int64_t e = (int64_t)r * cr + b;
        double re, im;
        if (h->prec == LEMPS_FP64) {
          const double* p = (const double*)buf.data();
          re = p[2 * e]; im = p[2 * e + 1];
        } else {
          const float* p = (const float*)buf.data();
          re = p[2 * e]; im = p[2 * e + 1];
        }
        tensors[2 * out] = re;
        tensors[2 * out + 1] = im;
        ++out;
      }
  }
  return LEMPS_OK;
}

lemps_status sim_sync(lemps_handle h) {
  if (!h) return fail(LEMPS_EINVAL, "sim_sync: null handle");
  if (h->sticky) return fail(LEMPS_ECUDA, "sim_sync: sticky CUDA error");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "sim_sync");
  std::vector<int32_t> st(h->B);
  if (cudaMemcpy(st.data(), h->status, sizeof(int32_t) * h->B, cudaMemcpyDeviceToHost) != cudaSuccess)
    return check_cuda(h, "sim_sync");
  for (auto v : st)
    if (v) return fail(LEMPS_ENUMERIC, "sim_sync: a trajectory flagged a numerical failure");
  return LEMPS_OK;
}

lemps_status sim_profile(lemps_handle h, int32_t enable, double* ms, int64_t* launches) {
  if (!h) return fail(LEMPS_EINVAL, "sim_profile: null handle");
  if (ms || launches) {
    h->collect_profile();
    for (int k = 0; k < LEMPS_NUM_KERNEL_KINDS; ++k) {
      if (ms) ms[k] = h->prof_ms[k];
      if (launches) launches[k] = h->prof_n[k];
    }
  }
  if (enable && !h->profiling) {
    h->collect_profile();
    for (int k = 0; k < LEMPS_NUM_KERNEL_KINDS; ++k) { h->prof_ms[k] = 0.0; h->prof_n[k] = 0; }
  }
  h->profiling = enable != 0;
  return check_cuda(h, "sim_profile");
}

lemps_status sim_tiles(lemps_handle h, int32_t* tile_m, int32_t* tile_n, double* tune_ms) {
  if (!h || !tile_m || !tile_n) return fail(LEMPS_EINVAL, "sim_tiles: null argument");
  const int np = h->n - 1;
  for (int kind = 0; kind < 3; ++kind)
    for (int q = 0; q < np; ++q) {
      const int id = h->tile_of(kind, q);
      int bm = 0, bn = 0;
      if (id >= 0) tile_shape(h->prec, id, bm, bn);
      tile_m[kind * np + q] = bm;
      tile_n[kind * np + q] = bn;
    }
  if (tune_ms) *tune_ms = h->tune_ms;
  return LEMPS_OK;
}

lemps_status destroy(lemps_handle h) {
  if (!h) return fail(LEMPS_EINVAL, "destroy: null handle");
  cudaStreamSynchronize(h->stream);
  h->collect_profile();
  h->release();
  delete h;
  return LEMPS_OK;
}

}  // extern "C"
