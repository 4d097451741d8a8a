// helk_internal.cuh -- shared declarations of the sm_103a HELIOS-K library.
//
// Device data layout (HBM):
//   line list  SoA doubles, ordered by nu0 (stable), one array per field.
//   LineRec64  64-byte per-line record of one (T, P) condition (FP64 form).
//   LineRec32  48-byte per-line record (FP32 form), strengths scaled by 2^-E.
//   ckey       per-line floor((nu0 - nu_min)/dnu) as double; non-decreasing
//              in list order, used to map grid tiles to line ranges.
//   kappa      doubles on the uniform grid.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/helk.h"

// Line-record budget of one chunk of helk_opacity_batch (64 GiB).
constexpr int64_t HELK_DEFAULT_BATCH_BUDGET = (int64_t)64 << 30;

namespace helk {

// ------------------------------------------------------------ constants --
// CGS; CODATA 2018 exact SI values.  T0 = 296 K (Sec. 2.3).
constexpr double KB = 1.380649e-16;       // erg / K
constexpr double CLIGHT = 2.99792458e10;  // cm / s
constexpr double AMU = 1.66053906660e-24; // g
constexpr double C2 = 1.4387768775039338021;  // h c / k_B [cm K]
constexpr double T0 = 296.0;
constexpr double PI = 3.1415926535897932384626;
constexpr double LN2 = 0.69314718055994530941723;
constexpr double SQRTLN2 = 0.83255461115769775635316;    // sqrt(ln 2)
constexpr double SQRTLN2PI = 0.46971863934982566688617;  // sqrt(ln 2 / pi)
constexpr double SQRTPI = 1.7724538509055160272982;
constexpr double INV_SQRTPI = 0.56418958354775628694808;
constexpr double ASINH_XCORE = 2.99822295029796973884;  // asinh(10): the surrogate's |x| feature scale
constexpr double GH3_T = 1.2247448713915890490986;       // sqrt(3/2)
// Region thresholds on r^2 = a^2 + u^2 (Sec. 2.4)
constexpr double R2_GH3 = 100.0;
constexpr double R2_GH1 = 1.0e6;
// Algorithm 916 series step and tail width: terms with |n h -+ x| > A916_TAIL
// are below e^{-38} of the largest one and are skipped.
constexpr double A916_H = 0.5;
constexpr double A916_TAIL = 6.2;
constexpr int A916_S1_TERMS = 13;  // e^{-(nh)^2} < 1e-18 beyond n = 13

// ------------------------------------------------------------ records ---
struct __align__(16) LineRec64 {
  double nu0p;     // shifted centre nu0 + delta P
  double ku;       // sqrt(ln2) / Gamma_D
  double a;        // damping sqrt(ln2) Gamma_L / Gamma_D
  double a2;       // a*a (rounded once, as the oracle does)
  double Sp;       // S sqrt(ln2/pi) / Gamma_D
  double erfcx_a;  // erfcx(a) (core region only; 0 if a >= 10)
  double sig1;     // sum_n e^{-(nh)^2}/((nh)^2 + a^2) (core region only)
  int32_t ilo, ihi;  // window, empty when ilo > ihi
};
static_assert(sizeof(LineRec64) == 64, "LineRec64 must be 64 bytes");

struct __align__(16) LineRec32 {
  int32_t c;       // reference grid index near the shifted centre
  int32_t ilo, ihi;
  float phi_k;     // (nu0' - nu_c) * ku: u_i = (i - c) beta - phi_k
  float beta;      // dnu * ku
  float a;         // damping
  float a2;        // a*a
  float P1;        // Sp a / sqrt(pi)      (scaled)   GH1 numerator
  float P3;        // Sp a (sqrt(pi)/6)/pi (scaled)   GH3 numerator
  float Sp;        // Sp                   (scaled)   core region
  float erfcx_a;   // erfcx(a)
  float sig1;      // core series S1(a)
};
static_assert(sizeof(LineRec32) == 48, "LineRec32 must be 48 bytes");

// Device-side error flags and upload checks.
struct DevStats {
  int err_flags;                    // ERRF_*
  int bad_lines;                    // validation failures at upload
  int unsorted;                     // upload: nu0 not ordered
  unsigned int tile_counter;        // next (condition, tile) item of the persistent Voigt kernel
};

// Core evaluations routed to the surrogate by the FP32 Voigt kernel: the
// kernel appends (grid point, condition, scaled S', x, y); entries past
// `cap` are evaluated in place by Algorithm 916 instead.
struct SurrQueue {
  unsigned long long count;  // 64-bit: a batch call may route more than 2^32 evaluations
  unsigned long long cap;
  int32_t *idx, *cond;
  float *w, *x, *y;
  const uint32_t *mask;  // validated cells of the network, nx * ny bits
  int nx, ny;
};

// One (T, P) condition of a call.
struct CondArgs {
  double T, P, q_ratio, pad;
};

// Per-condition results of line preparation and of the Voigt kernel.
struct CondStats {
  unsigned long long evals;         // sum of window sizes
  unsigned long long region[4];     // evaluations per method (optional):
                                    // [916, GH3, GH1, 916 series terms]
  long long wmax;                   // max half-width of a window in points (-1: none)
  unsigned long long spmax_bits;    // max S' (non-negative double bits)
  int scale_exp;                    // FP32 form: strengths scaled by 2^-scale_exp
  int core_w1;                      // FP32 form: 1 + max distance (points) from a line's
                                    // reference index to a point of its core, 0: no core
};
// Kernel-side error flags (DevStats::err_flags), reported by helk_sync:
//   ERRF_TIMEOUT    a bounded wait gave up
//   ERRF_F32_RANGE  a line's core lies beyond 2^23 grid points of its centre,
//                   where the FP32 form's point offsets are no longer exact
enum { ERRF_TIMEOUT = 1, ERRF_F32_RANGE = 2 };

// FP32 form: grid points per block of the per-block core reach (the largest
// distance from a line's reference index to a point of its core, over the
// lines whose reference index lies in the block), which bounds the candidate
// lines of the core kernel's warps.
constexpr int CORE_BLK_PTS = 4096;  // 2^12 (k_pack32 takes the block by a shift)
__host__ __device__ inline int core_blocks(int64_t ngrid) { return (int)((ngrid + CORE_BLK_PTS - 1) / CORE_BLK_PTS); }

// ---------------------------------------------------------- the context --
}  // namespace helk

struct helk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int num_sms = 0;
  int max_smem_optin = 0;
  // line list (sorted SoA)
  int64_t nlines = 0;
  bool has_E = false, has_gself = false, has_ncoll = false, has_delta = false;
  bool has_mass = false, has_weight = false;
  double *nu0 = nullptr, *S0 = nullptr, *El = nullptr, *gair = nullptr,
         *gself = nullptr, *ncoll = nullptr, *delta = nullptr, *lmass = nullptr,
         *lweight = nullptr;
  int64_t lines_cap = 0;
  // per-call scratch
  helk::LineRec64 *rec64 = nullptr;
  int64_t launches = 0;  // kernels this context has launched (for tracing)
  helk::LineRec32 *rec32 = nullptr;
  int2 *core_rng = nullptr;  // FP32 form: each line's core points [x, y] (x > y: none)
  int64_t core_cap = 0;
  int *core_blk = nullptr;   // FP32 form: 1 + core reach per block of CORE_BLK_PTS points, per condition
  int64_t core_blk_cap = 0;
  double *ckey = nullptr;
  int64_t ckey_cap = 0;
  int32_t *ckey32 = nullptr;  // FP32 form: ckey clamped to the int32 range (order kept), for integer searches
  int64_t ckey32_cap = 0;
  // FP32 form: the core kernel runs on side_stream beside the main Voigt
  // kernel and leaves its per-point sums in kcore (FP32, n_cond x n points)
  float *kcore = nullptr;
  int64_t kcore_cap = 0;
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int64_t rec_cap = 0, rec32_cap = 0;
  int32_t *tile_lo = nullptr, *tile_hi = nullptr;
  int64_t tile_cap = 0;
  helk::DevStats *stats = nullptr;      // device
  helk::DevStats *stats_host = nullptr; // pinned
  // conditions of the current call
  helk::CondArgs *cond_dev = nullptr, *cond_host = nullptr;  // host side pinned
  helk::CondStats *cstats = nullptr, *cstats_host = nullptr; // host side pinned
  int *cond_order = nullptr;
  int cond_cap = 0;
  int last_ncond = 0;
  cudaEvent_t cond_ev = nullptr;   // completion of the last batch that read cond_host
  // CUDA graph of the batched path
  cudaStream_t cap_stream = nullptr;
  std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;  // by call shape, oldest first
  // line-record bytes one chunk of a batch may use (helk_set_batch_budget)
  int64_t batch_budget = HELK_DEFAULT_BATCH_BUDGET;
  // opacity output owned by the context
  double *kappa = nullptr;
  int64_t kappa_cap = 0;
  int64_t last_n = 0;
  bool have_opacity = false;
  bool last_counted_regions = false;
  // k-distribution scratch
  unsigned long long *sort_a = nullptr, *sort_b = nullptr;
  int64_t sort_cap = 0;
  double *pinv = nullptr;  // pseudo-inverse of the Chebyshev design matrix
  int64_t pinv_cap = 0, pinv_nb = 0;
  int pinv_ncheb = 0;
  // fit stage: logarithm pairs, partial sums, per-row counts of finished
  // CTAs (zero between calls)
  void *kd_fold = nullptr, *kd_part = nullptr, *kd_done = nullptr;
  int64_t kd_fold_cap = 0, kd_part_cap = 0, kd_done_cap = 0;
  double *coef_dev = nullptr, *mean_dev = nullptr;
  int64_t coef_cap = 0, mean_cap = 0;
  // Voigt surrogate network (k_mlp.cu): FP32 parameters, Adam moments,
  // gradient, training set, validated-cell mask
  float *mlp_p = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_g = nullptr, *mlp_loss = nullptr;
  int mlp_step = 0;
  float *mlp_feat = nullptr, *mlp_tgt = nullptr;
  int64_t mlp_data_cap = 0;
  uint32_t *mlp_mask = nullptr;  // bit c of word c/32: cell c validated
  int mlp_mask_nx = 0, mlp_mask_ny = 0;
  // queue of core evaluations routed to the network
  helk::SurrQueue *squeue = nullptr;  // device struct
  void *squeue_buf = nullptr;
  int64_t squeue_cap = 0;
  // column masses of helk_transmission
  double *mass_col = nullptr;
  int64_t mass_col_cap = 0;
  // transmission: the bins' differences as scaled pairs, per-bin constants
  void *tr_pairs = nullptr, *tr_bins = nullptr;
  int64_t tr_pairs_cap = 0, tr_bins_cap = 0;
  // generic upload scratch
  void *tmp = nullptr;
  int64_t tmp_cap = 0;
  // autotuned Voigt kernel shape code per precision (0 = heuristic), valid for
  // grids of tuned_n points
  int tuned_tile[2] = {0, 0};
  int64_t tuned_n[2] = {0, 0};
  // stage timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev[HELK_NSTAGES];  // start/end pairs
  int64_t ev_used[HELK_NSTAGES] = {0, 0, 0, 0};
  bool ev_overflow[HELK_NSTAGES] = {false, false, false, false};
};

namespace helk {

// ------------------------------------------------------------- helpers --
// Stage timing: record the start / end event of one stage launch.
void stage_begin(helk_ctx *c, int stage);
void stage_end(helk_ctx *c, int stage);
helk_status set_err(helk_ctx *c, helk_status st, const std::string &msg);
helk_status cuda_check(helk_ctx *c, cudaError_t e, const char *what);
// Grow a device buffer to at least `bytes` (contents are not kept).
helk_status ensure_buf(helk_ctx *c, void **p, int64_t *cap_bytes, int64_t bytes,
                       const char *what);

// Nanoseconds of the GPU's global timer (it keeps running while a kernel
// waits or is preempted).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: polls mbarrier.try_wait (which may
// suspend the thread for a while on each poll) until the phase completes or
// `limit_ns` nanoseconds of the global timer have passed since the first
// failed poll; then sets ERRF_TIMEOUT in *flags and returns false.  The bound
// is in time, not in polls, so it holds whatever a poll's suspension costs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar_smem, uint32_t parity, int *flags,
                                                  unsigned long long limit_ns) {
  bool started = false;
  unsigned long long t0 = 0;
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar_smem), "r"(parity)
        : "memory");
    if (done) return true;
    const unsigned long long t = global_ns();
    if (!started) {
      started = true;
      t0 = t;
    } else if (t - t0 >= limit_ns) {
      atomicOr(flags, ERRF_TIMEOUT);
      return false;
    }
  }
}

// The lanes of the warp whose 8-bit digit equals this lane's (what a
// match-any over the digit gives), from eight ballots, one per digit bit: a
// fixed cost, where a match-any's cost grows with the number of distinct
// values among the lanes.  Lanes with valid == false match no lane; their
// own result is their own bit.
__device__ __forceinline__ uint32_t warp_digit_peers(uint32_t d, bool valid) {
  uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t m = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? m : ~m;
  }
  return valid ? peers : (1u << (threadIdx.x & 31));
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 1-D bulk TMA copy global -> shared, completing on an mbarrier.  dst, src
// 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(uint32_t dst_smem, const void *src, uint32_t bytes,
                                            uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst_smem),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// ---------------------------------------------------------- launchers ---
// k_lines.cu
cudaError_t launch_validate_lines(helk_ctx *c, int64_t n);
cudaError_t launch_sort_lines(helk_ctx *c, int64_t n);  // orders SoA by nu0
// n_cond conditions: from c->cond_dev, or (n_cond == 1 and single != NULL)
// the one condition passed by value.  Records of condition k start at
// k * nlines; tile maps at k * ntiles.
// a916_f64: also the FP64 Algorithm 916 per-line factors (erfcx(a), S1(a)),
// which only the FP64 form reads.
cudaError_t launch_lineprep(helk_ctx *c, int n_cond, const CondArgs *single, double mass,
                            const helk_cutoff &cut, const helk_grid &g, bool a916_f64);
cudaError_t launch_pack32(helk_ctx *c, int n_cond, const helk_grid &g);
cudaError_t launch_tilemap(helk_ctx *c, int n_cond, const helk_grid &g, int tile, int64_t ntiles);
// Conditions ordered by decreasing evaluation count (largest work first).
cudaError_t launch_cond_order(helk_ctx *c, int n_cond);
// k_voigt.cu
// Voigt kernel shapes.  A shape code names one built configuration of a
// precision's kernel (FP32: the 1-based position in its shape list; FP64:
// the slots per warp, 1..8).  voigt_shape_info gives the shape's tile
// (points per CTA), warps per CTA and candidate lines per pipeline stage,
// or returns false for an unknown code.
bool voigt_shape_info(int precision, int code, int *points, int *warps, int *lines_per_stage);
// The shape for a grid of n points (the tuned one, else one whose tile count
// fills whole waves of resident CTAs).
int voigt_shape(helk_ctx *c, int precision, int count, int64_t n);
// Shape codes the autotuner times.
int voigt_shape_candidates(int precision, int *out, int max);
// Persistent Voigt kernel over n_cond x ntiles (condition, tile) items taken
// from DevStats::tile_counter (reset to 0 before the launch); kappa of
// condition k at kappa + k * g.n.
cudaError_t launch_voigt(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o,
                         double *kappa, int shape, int64_t ntiles);
// FP32 form: the Algorithm 916 cores that k_voigt_f32 leaves out, added into
// kappa (launched after launch_voigt; no-op for the FP64 form).
cudaError_t launch_voigt_core(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o);
cudaError_t launch_core_add(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o, double *kappa);
// k_voigt64.cu: the FP64 form (called by the dispatch above) and the
// bounded-wait self-test
bool f64_shape_info(int code, int *points, int *warps, int *lines_per_stage);
int f64_shape_candidates(int *out, int max);
int f64_shape(helk_ctx *c, int count, int64_t n);
cudaError_t launch_voigt_f64(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o, double *kappa,
                             int shape, int64_t ntiles);
cudaError_t launch_selftest_timeout(helk_ctx *c, int limit_us);
// k_kdist.cu
int64_t pinv_bytes(int64_t nb, int ncheb);
int64_t pinv_work_doubles(int64_t nb, int ncheb);
cudaError_t launch_pinv(helk_ctx *c, int64_t nb, int ncheb, double *work);
cudaError_t launch_kdist_bins(helk_ctx *c, const double *kappa, int64_t n, int nbins, int ncheb,
                              double kappa_floor, double *coef, double *mean, double *kg_out);
int64_t kdist_smem_max_points(helk_ctx *c);
// scratch of the fit stage: folded logarithms, per-group partial sums
int64_t kdist_fold_bytes(int64_t n, int nbins);
int64_t kdist_part_bytes(helk_ctx *c, int64_t n, int nbins);
int64_t kdist_done_bytes(int nbins);
size_t trans_pair_bytes(int nbins, int64_t nb);
size_t trans_bin_bytes(int nbins);
// k_mlp.cu
constexpr int MLP_NPARAMS_H = 8577;
cudaError_t launch_mlp_eval(helk_ctx *c, const float *params, int64_t n, const double *x, const double *y,
                            double *k);
cudaError_t launch_mlp_train_step(helk_ctx *c, const float *params, const float *feat, const float *tgt,
                                  int64_t b0, int64_t B, float *grads, float *loss);
cudaError_t launch_mlp_adam(helk_ctx *c, float *p, float *m, float *v, const float *grad, float lr, int step);
cudaError_t launch_mlp_samples(helk_ctx *c, int64_t n, uint64_t seed, float *feat, float *tgt, double *xs,
                               double *ys);
cudaError_t launch_a916_points(helk_ctx *c, int64_t n, const double *x, const double *y, double *k);
cudaError_t launch_mlp_validate(helk_ctx *c, int nx, int ny, int per_cell, double *err_dev);
cudaError_t launch_mlp_queue(helk_ctx *c, int n_cond, int64_t ngrid, double weight, double *kappa);
// k_probe.cu: throughput probes (kind: HELK_PROBE_*); sink holds `blocks`
// doubles
cudaError_t launch_probe(helk_ctx *c, int kind, int iters, int blocks, void *sink);
int probe_blocks(helk_ctx *c);
int probe_ops_per_iter();
int probe_threads();
cudaError_t launch_transmission(helk_ctx *c, int nbins, int64_t nb, const double *sorted,
                                const double *coef, int ncheb, int ng, int nm, const double *m_dev,
                                double *direct, double *fit);

}  // namespace helk
