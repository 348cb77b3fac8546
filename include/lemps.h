/*
 * lemps.h — C ABI of the GB300 library for batched Monte-Carlo MPS
 * trajectories with the locally entanglement-optimal unraveling
 * (arXiv 2508.05745).
 *
 * The problem statement follows Sec. III (truncated trajectory sampling of a
 * circuit description D = initial state |0...0>, a string of layers of
 * nearest-neighbour two-qubit gates, each followed by single-qubit noise on the
 * two gated qubits) and Sec. IV (the MPS update of Sec. IV.A, the channel
 * unraveling subprocedure of Alg. 1, the optimal Kraus set of Sec. IV.B).
 *
 * Conventions shared by every call
 *  - Complex numbers are interleaved (re, im) doubles.
 *  - A two-qubit gate on qubits (q, q+1) is a row-major 4x4 matrix indexed by
 *    2*s_q + s_{q+1}; a Kraus operator is a row-major 2x2 matrix K[s'][s].
 *  - Pointers documented as "host" are caller-owned and only read (or written)
 *    during the call.  Pointers documented as "device" must point to memory on
 *    the handle's (or the given stream's) device.
 *  - Functions never throw and never fall back to the CPU.  A non-OK status
 *    leaves the handle usable, except LEMPS_ECUDA, which is sticky: every later
 *    call on that handle returns LEMPS_ECUDA.  lemps_last_error() describes the
 *    last failure of the calling thread.
 *  - Random numbers: the uniform of slot s (0 = qubit q, 1 = qubit q+1, 2 = the
 *    per-gate noise coin) of global gate g in trajectory t is
 *    Philox4x64-10(counter = (t, g, s, 0), key = (seed, 0x4C454D5053545241)),
 *    first output word >> 11, times 2^-53.  Results therefore do not depend on
 *    how trajectories are batched or sharded (traj_offset).
 *  - Runs are deterministic: each trajectory is computed by its own thread
 *    blocks with a fixed order of operations (the eigensolver's shared sums
 *    are exact fixed-point integer adds), so the same configuration and calls
 *    give the same results bit for bit, whatever the batch, the wave size or
 *    the GEMM tile setting.
 */
#ifndef LEMPS_H
#define LEMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lemps_sim* lemps_handle;

typedef enum {
  LEMPS_OK = 0,
  LEMPS_EINVAL = 1,    /* invalid argument; nothing was enqueued */
  LEMPS_ENOMEM = 2,    /* device allocation failed */
  LEMPS_ECUDA = 3,     /* CUDA error; sticky */
  LEMPS_ENUMERIC = 4,  /* a trajectory produced NaN / lost its norm / eigensolver cap */
  LEMPS_ESTATE = 5     /* call not valid in the handle's current state */
} lemps_status;

typedef enum {
  LEMPS_FP64 = 0,      /* complex128 storage and arithmetic everywhere */
  LEMPS_MIXED = 1      /* complex64 MPS storage and contractions (two-site
                          tensor, Gram matrix, projections, centre moves);
                          the Gram eigensolve of the split (tridiagonal form,
                          eigenvalues, tridiagonal eigenvectors), reduced
                          densities, unraveling, branch weights, discarded
                          weights and entropies in FP64 (complex128); the
                          kept eigenvectors are back-transformed in complex64,
                          the precision they are used in */
} lemps_precision;

typedef enum {
  LEMPS_UNRAVEL_OPTIMAL = 0,  /* remix each noise site's Kraus set into the
                                 locally entanglement-optimal one (Sec. IV.B) */
  LEMPS_UNRAVEL_GIVEN = 1,    /* sample the Kraus set as given (fixed
                                 unravelings such as Orthogonal or Projective,
                                 Sec. V.A and the appendix on common unravelings) */
  LEMPS_UNRAVEL_HAAR_OPT = 2  /* "Haar Optimal" fixed unraveling (Sec. V.B,
                                 near-optimal fixed unraveling for random
                                 circuits): the Kraus set is remixed once into
                                 the locally entanglement-optimal set for the
                                 Bell state (reduced state I/2), which by the
                                 least-unitary corollary is also the decomposition
                                 of least average unitarity, and then sampled as
                                 given at every site */
} lemps_unravel;

typedef enum {
  LEMPS_LAYER_LOCAL = 0,  /* gate, its noise, truncation of its bond, gate by
                             gate: (Trunc N^{(x)2} U)^{(x) n/2} (Sec. IV.A,
                             layering options) */
  LEMPS_LAYER_GLOBAL = 1  /* all gates of the layer, then the noise on every
                             gated pair in gate order, then every bond
                             truncated to chi_max by a left-to-right sweep:
                             Trunc^{(x) n-1} N^{(x) n} U^{(x) n/2} (Sec. IV.A).
                             Bonds reach 2 chi_max inside a layer, so chi_max
                             is limited to 64; lower discarded weight */
} lemps_layering;

/* Device allocator hook (PyTorch's caching allocator from Python).  NULL
 * alloc means cudaMalloc / cudaFree.  Blocks must be 16-byte aligned (the
 * kernels stream workspaces with bulk copies); sim_create fails with
 * LEMPS_EINVAL on a misaligned block. */
typedef void* (*lemps_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*lemps_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct {
  int32_t n_qubits;       /* >= 2 */
  int32_t chi_max;        /* maximum bond dimension, 1..512 (above 128 the
                             centre moves and eigensolves of sites whose
                             capacity exceeds 128 run unblocked kernels that
                             keep their matrices in global memory: Gram
                             matrices up to 1024; sample_bitstrings then needs
                             chi_max <= 256) */
  double trunc_cutoff;    /* keep Schmidt weights > cutoff * total (Sec. II truncation) */
  int64_t n_traj;         /* trajectories held by this handle */
  int64_t traj_offset;    /* global id of the handle's first trajectory */
  uint64_t seed;
  int32_t precision;      /* lemps_precision */
  int32_t unravel_mode;   /* lemps_unravel */
  int32_t log_capacity;   /* gates whose sampled branch indices are kept (sample_branch) */
  double eps_max;         /* per-trajectory error cap of Thm. 1 (App. B), >= 2 */
  void* cuda_stream;      /* cudaStream_t used by every call, NULL = default stream */
  lemps_alloc_fn alloc;
  lemps_free_fn free;
  void* alloc_ctx;
  int32_t layering;       /* lemps_layering (0 = local) */
  int64_t max_traj_in_flight; /* trajectories held on the device at once (a
                             wave); 0 = automatic: as many as fit in 60 % of the
                             device memory (and 90 % of what is free).  When
                             n_traj exceeds it, the handle runs in waves (see
                             measure) */
  int32_t eigvec_fp64;    /* LEMPS_MIXED only: 1 = back-transform the kept
                             eigenvectors of the split in FP64 as well (FP64-
                             accurate eigenpairs, rounded to complex64 when the
                             split uses them); 0 = back-transform them in
                             complex64, the precision they are used in (the
                             eigenvalues, the truncation and the tridiagonal
                             eigenvectors are FP64 either way) */
  int32_t gemm_tile;      /* output tile (rows x columns) of the SIMT GEMMs of
                             the two-site contraction and of the Gram matrix:
                             0 = picked per problem size by the autotuner of
                             sim_create (see sim_tiles); 1..4 = fixed shape:
                             complex128 64x64, 32x64, 64x32, 32x32; complex64
                             64x64, 128x64, 64x128, 32x32.  Every shape gives
                             the same results bit for bit */
  int32_t big_kernels;    /* 0 = the centre moves and eigensolves run the
                             global-memory kernels only where a site capacity
                             exceeds 128 (their on-chip counterparts stop
                             there); 1 = everywhere (slower; a check of those
                             kernels against the oracle on small cases) */
} lemps_config;

typedef struct {
  int32_t n_gates;            /* gates of this layer, applied in list order */
  const int32_t* left_qubit;  /* host [n_gates]; gate k acts on (q, q+1), pairs disjoint */
  const double* gates;        /* host [n_gates][4][4] complex */
  int32_t n_kraus;            /* operators of the single-qubit noise channel: 1..4
                                 for the optimal and Haar-optimal modes, 1..8 for
                                 LEMPS_UNRAVEL_GIVEN (e.g. the 5-operator
                                 Projective depolarizing set) */
  const double* kraus;        /* host [n_kraus][2][2] complex, sum K^dagger K = I */
  double coin_p;              /* the channel acts on both gated qubits with this
                                 probability per gate (1 = always) */
} lemps_layer;

typedef struct {
  /* per-trajectory outputs, host, optional (NULL = not returned) */
  double* z;           /* [n_traj][n]     <Z_i> */
  double* zz;          /* [n_traj][n-1]   <Z_i Z_{i+1}> */
  double* s_half;      /* [n_traj]        entropy (nats) of bond n/2 */
  double* eps_bound;   /* [n_traj]        error bound of Thm. 1 / App. B */
  int32_t* status;     /* [n_traj]        0 = ok, else OR of LEMPS_ENUMERIC reason bits:
                                          1 NaN/Inf, 2 lost norm, 4 eigensolver cap,
                                          8 shape (internal), 16 copy time limit (internal) */
  /* reductions over trajectories, host, required */
  double* z_mean;      /* [n] */
  double* z_stderr;    /* [n] */
  double* zz_mean;     /* [n-1] */
  double* zz_stderr;   /* [n-1] */
  double s_half_mean;
  double s_half_stderr;
  double eps_hat;      /* mean eps_bound */
  double eps_buffer;   /* sqrt(eps_max^2 / (2N) ln(1/delta)), delta = 0.05 */
  int64_t n_failed;    /* trajectories with a non-zero status */
} lemps_measurement;

/* Allocate a batch of n_traj trajectories in |0...0> (all bonds 1).  All
 * device memory is owned by the handle. */
lemps_status sim_create(const lemps_config* cfg, lemps_handle* out);

/* Apply one layer (Sec. IV.A, layering option "local", Trunc o N(x)N o U per
 * gate) to every trajectory: contract the gate into the two-site tensor,
 * unravel the noise on q then q+1 (Alg. 1 with the Kraus set of Sec. IV.B),
 * sample with the Philox stream above, re-split by a Hermitian eigensolve of
 * the two-site Gram matrix and truncate to chi_max.  Asynchronous on the
 * handle's stream; the host arrays are copied before return. */
lemps_status apply_layer(lemps_handle h, const lemps_layer* layer);

/* Standalone optimal unraveling (Sec. IV.B, App. F.2) of a batch of target
 * reduced states.  rho_a: device [batch][2][2] complex (Hermitian, any trace);
 * kraus: device [n_kraus][2][2] complex (n_kraus 1..4); kraus_out: device
 * [batch][4][2][2] complex, kraus_out[b][k] = sum_j W[j][k] K_j; e_av: device
 * [batch] ensemble-averaged entropy (nats) of the output set on rho_a/Tr.
 * Asynchronous on stream. */
lemps_status unravel_opt(const double* rho_a, const double* kraus, int32_t n_kraus, int64_t batch,
                         double* kraus_out, double* e_av, void* stream);

/* Branch indices sampled at global gate index `gate` (slot 0: qubit q, 1:
 * qubit q+1) for every trajectory; -1 where the noise coin skipped the gate.
 * branch_out: host [n_traj].  Synchronizes the stream. */
lemps_status sample_branch(lemps_handle h, int64_t gate, int32_t slot, int32_t* branch_out);

/* Observables of Sec. III.C / App. C on the current states, mean and standard
 * error over trajectories, and the a-posteriori error estimate of Thm. 1.
 * Moves every trajectory's orthogonality centre; synchronizes the stream.
 * Waves (n_traj > max_traj_in_flight): trajectories are independent (Sec.
 * III), so one wave of at most max_traj_in_flight trajectories is resident
 * on the device; apply_layer advances it and keeps a host copy of every
 * layer.  measure measures the resident wave, then puts each other wave in
 * |0...0> and brings it through the recorded layers before measuring it
 * (global trajectory ids, so the results equal those of one big handle:
 * per trajectory bit for bit, means and standard errors merged exactly up to
 * rounding); the last wave processed stays resident.  The per-trajectory
 * outputs cover all n_traj trajectories.  sample_branch, sample_bitstrings,
 * eps_concentrated and sim_export_mps need a single wave (LEMPS_ESTATE
 * otherwise); sim_sync checks the resident wave. */
lemps_status measure(lemps_handle h, lemps_measurement* m);

/* The wave size (trajectories held on the device) and the number of waves of
 * the handle. */
lemps_status sim_waves(lemps_handle h, int64_t* wave_size, int32_t* n_waves);

/* Output-distribution sampling (Lemma sampling_reduction; Corollary on output
 * distribution sampling): draws n_shots (1..65535) computational-basis
 * bitstrings from every trajectory's current MPS by sequential conditional
 * sampling over the sites, qubit 0 first; over trajectories they sample the
 * unraveled mixed state.  bits_out: host [n_traj][n_shots][n] bytes 0/1.
 * Random numbers: Philox counter (trajectory id, 2^62 + shot, site, 0), a
 * domain the noise sites never use.  Moves the orthogonality centre to site
 * 0; keeps one device buffer of the largest request (through the handle's
 * allocator); synchronizes the stream.  LEMPS_EINVAL when chi_max > 256. */
lemps_status sample_bitstrings(lemps_handle h, int32_t n_shots, uint8_t* bits_out);

/* Concentration-improved error bound (Sec. III.C; appendix on concentration
 * bounds): per trajectory sum_l w(L - l) eps_approx(l) over the L layers
 * applied so far, eps_approx(l) = 4 sqrt(2 sum of the layer's discarded
 * weights), with w(k) = alpha^k (kind 0, param = alpha in (0, 1]; alpha = 1
 * gives the plain bound of Thm. 1) or min(sqrt(8 n) (1 - p)^k, 1) for local
 * depolarizing noise of rate p (kind 1, param = p).  Capped like the plain
 * bound (kept when <= eps_max - 2, else eps_max).  eps_out: host [n_traj],
 * optional; eps_hat receives the mean.  The per-layer history holds 256
 * layers: LEMPS_ESTATE after more.  Synchronizes the stream. */
lemps_status eps_concentrated(lemps_handle h, int32_t kind, double param, double* eps_out, double* eps_hat);

/* Copy trajectory `traj`'s MPS to the host: bond_dims [n+1]; tensors receives
 * site k as [d_k][2][d_{k+1}] complex, sites concatenated (caller sizes it for
 * n * 2 * chi_max^2 complex).  Inspection only; synchronizes the stream. */
lemps_status sim_export_mps(lemps_handle h, int64_t traj, int32_t* bond_dims, double* tensors);

/* Wait for the handle's queued work; returns the sticky status and reports
 * LEMPS_ENUMERIC if any trajectory flagged a numerical failure. */
lemps_status sim_sync(lemps_handle h);

/* Release every device allocation of the handle. */
lemps_status destroy(lemps_handle h);

/* Expected branch entropy of a remixed Kraus set and its gradient (the
 * differentiation workload; cost of Eq. target_optimal_unitary, remix
 * K'_k = sum_j U[j][k] K_j with U = exp(iH), Eq. unitarity_kraus).
 *   theta:  device [batch][chi][2][2][chi] complex, double (theta_fp64 = 1) or
 *           float (0); target = first physical index; any norm.
 *   p:      device [batch] depolarizing rates of the channel being remixed
 *           (Kraus set {sqrt(1-3p/4) I, sqrt(p)/2 X, Y, Z}).
 *   h:      device [batch][4][4] complex Hermitian, read.
 *   cost:   device [batch], E(H) in nats.
 *   grad:   device [batch][4][4] complex Hermitian gradient Gamma with
 *           dE = Re Tr(Gamma^dagger dH), or NULL.
 *   rho_out: device [batch][2][2] complex reduced target states, or NULL.
 * Asynchronous on stream. */
lemps_status unravel_grad(const void* theta, int32_t theta_fp64, int64_t batch, int32_t chi,
                          const double* p, const double* h, double* cost, double* grad,
                          double* rho_out, void* stream);

/* `steps` gradient-descent steps H <- H - alpha * Gamma on the device (the
 * per-site unraveling optimisation of the differentiation workload, driving
 * the cost of Eq. target_optimal_unitary towards its minimum E_oF of Thm. 2)
 * for the reduced states rho_a (device [batch][2][2] complex, e.g. rho_out
 * above).  The step size is found by backtracking: it starts at lr, is halved
 * until E(H - alpha Gamma) <= E(H) - 1e-4 alpha ||Gamma||_F^2 (the step is
 * skipped once alpha < 1e-12), and the next step starts from twice the final
 * alpha (at most 1e4).  h is updated in place; cost_trace: device
 * [steps][batch] costs after each step, or NULL. */
lemps_status unravel_descend(const double* rho_a, const double* p, int64_t batch, int32_t steps,
                             double lr, double* h, double* cost_trace, void* stream);

/* Allocation-free variant of unravel_grad (the paper has no counterpart; it
 * is a service for callers that must not allocate device memory during a call:
 * code whose device memory is fully owned by another allocator, or latency
 * paths where cudaMalloc/cudaFree would synchronize the device).  Same
 * arguments and results as unravel_grad with rho_out = NULL, but the per-call
 * scratch (the reduced target states) lives in a static device array sized for
 * at most 16384 problems (1 MiB), which every GPU that loads the library holds
 * until the process exits.  batch > 16384 returns LEMPS_EINVAL.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, so make that first call before any stream capture.  The
 * address is kept for the life of the process: after a cudaDeviceReset (or
 * anything else that recreates the device's primary context) it is stale, so
 * do not call this entry point again on that device in the same process.  All
 * calls on one device share its copy of the array, which keeps the last call's
 * contents: calls that overlap on the same GPU (e.g. on different streams) race
 * and must be ordered by the caller.  No cudaMalloc, cudaFree or other
 * allocating routine is called. */
lemps_status unravel_grad_noalloc(const void* theta, int32_t theta_fp64, int64_t batch, int32_t chi,
                                  const double* p, const double* h, double* cost, double* grad, void* stream);

/* GEMM tile shapes of the handle (Sec. IV.A's contraction and Gram
 * products; the tile is an implementation choice the paper does not make).
 * Per gate position q = 0..n-2 (the pair (q, q+1)): row 0 of the outputs is
 * the two-site contraction, row 1 the Gram matrix of the left side (centre
 * moving right), row 2 that of the right side.  tile_m, tile_n: host [3][n-1],
 * the output tile's rows and columns, 0 where the tensor-core contraction runs
 * instead (mixed precision, site capacities 64..128).  tune_ms: host,
 * optional: milliseconds sim_create spent timing candidates.
 * Autotuning (gemm_tile = 0): for each kernel and each distinct triple of site
 * capacities (cap_q, cap_q+1, cap_q+2), sim_create times every candidate
 * shape on min(n_traj, 2 x the SM count) trajectories with every bond at its
 * capacity (capacity triples up to 128; larger ones keep 64x64) and zero operands (one warm-up and three timed launches, CUDA events
 * on the handle's stream, before the state is initialized) and keeps the
 * fastest; the default 64x64 stays unless another shape is at least 3 % faster.
 * The choice is kept per device and precision for the life of the process, so
 * later handles with the same capacities reuse it without timing.  Since every
 * shape gives the same results, the choice never changes an output. */
lemps_status sim_tiles(lemps_handle h, int32_t* tile_m, int32_t* tile_n, double* tune_ms);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch made by apply_layer (enable = 1 starts a fresh record,
 * enable = 0 stops recording).  With ms and launches non-NULL the call
 * synchronizes and returns, per kernel kind (LEMPS_K_*), the summed event
 * time in milliseconds and the launch count since recording started. */
enum {
  LEMPS_K_MOVE = 0,      /* centre move (Householder QR / LQ + merge) */
  LEMPS_K_CONTRACT = 1,  /* two-site contraction (tensor cores in mixed mode for
                            site capacities 64-128) + 4x4 reduced density */
  LEMPS_K_UNRAVEL = 2,   /* noise sites: optimal unraveling + sampling */
  LEMPS_K_GRAM = 3,      /* apply gate and Kraus operators, Gram matrix */
  LEMPS_K_EIG = 4,       /* Hermitian eigensolver: Householder tridiagonalization,
                            Sturm/Newton eigenvalues, inverse iteration,
                            back-transformation */
  LEMPS_K_SPLIT = 5,     /* truncation and new site tensors */
  LEMPS_K_OTHER = 6,     /* layer bookkeeping */
  LEMPS_NUM_KERNEL_KINDS = 7
};
lemps_status sim_profile(lemps_handle h, int32_t enable, double* ms, int64_t* launches);

const char* lemps_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LEMPS_H */
