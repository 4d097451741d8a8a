// helk_api.cu -- the C ABI (include/helk.h): argument checks, context-owned
// device buffers, and the order of kernel launches for each entry point.
#include <cuda_runtime.h>
#include <cmath>
#include <cstddef>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <string>

#include "helk_internal.cuh"

using namespace helk;

namespace helk {

helk_status set_err(helk_ctx *c, helk_status st, const std::string &msg) {
  if (c) c->err = msg;
  return st;
}

helk_status cuda_check(helk_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return HELK_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_err(c, HELK_ERR_OOM, std::string(what) + ": out of device memory");
  }
  return set_err(c, HELK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

helk_status ensure_buf(helk_ctx *c, void **p, int64_t *cap_bytes, int64_t bytes, const char *what) {
  if (bytes <= *cap_bytes && *p) return HELK_OK;
  if (*p) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, what);
    cudaFree(*p);
    *p = nullptr;
    *cap_bytes = 0;
  }
  int64_t alloc = bytes < 256 ? 256 : bytes;
  cudaError_t e = cudaMalloc(p, (size_t)alloc);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_check(c, e, what);
  }
  *cap_bytes = alloc;
  return HELK_OK;
}

constexpr int64_t EV_MAX_PAIRS = 65536;

void stage_begin(helk_ctx *c, int stage) {
  if (!c->profiling) return;
  auto &v = c->ev[stage];
  const int64_t i = c->ev_used[stage];
  if (i >= EV_MAX_PAIRS) {
    c->ev_overflow[stage] = true;
    return;
  }
  while ((int64_t)v.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      c->ev_overflow[stage] = true;
      return;
    }
    v.push_back(e);
  }
  cudaEventRecord(v[2 * i], c->stream);
}

void stage_end(helk_ctx *c, int stage) {
  if (!c->profiling || c->ev_overflow[stage]) return;
  const int64_t i = c->ev_used[stage];
  if (i >= EV_MAX_PAIRS || (int64_t)c->ev[stage].size() < 2 * (i + 1)) return;
  cudaEventRecord(c->ev[stage][2 * i + 1], c->stream);
  c->ev_used[stage] = i + 1;
}

}  // namespace helk

#define HELK_TRY(expr)              \
  do {                              \
    helk_status _s = (expr);        \
    if (_s != HELK_OK) return _s;   \
  } while (0)

static helk_status bind_device(helk_ctx *c) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != c->device) return cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice");
  return HELK_OK;
}

static bool is_fin(double v) { return std::isfinite(v); }

extern "C" {

helk_status helk_create(helk_ctx **out, int device, void *stream) {
  if (!out) return HELK_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return HELK_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return HELK_ERR_INVALID_ARG;
  helk_ctx *c = new (std::nothrow) helk_ctx();
  if (!c) return HELK_ERR_OOM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return HELK_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (cudaMalloc(&c->stats, sizeof(DevStats)) != cudaSuccess ||
      cudaMallocHost(&c->stats_host, sizeof(DevStats)) != cudaSuccess) {
    cudaGetLastError();
    helk_destroy(c);
    return HELK_ERR_OOM;
  }
  memset(c->stats_host, 0, sizeof(DevStats));
  if (cudaMemset(c->stats, 0, sizeof(DevStats)) != cudaSuccess) {
    helk_destroy(c);
    return HELK_ERR_CUDA;
  }
  *out = c;
  return HELK_OK;
}

void helk_destroy(helk_ctx *c) {
  if (!c) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->side_stream) cudaStreamSynchronize(c->side_stream);
  if (c->mass_col) cudaFree(c->mass_col);
  for (void *p : {(void *)c->mlp_p, (void *)c->mlp_m, (void *)c->mlp_v, (void *)c->mlp_g,
                  (void *)c->mlp_loss, (void *)c->mlp_feat, (void *)c->mlp_tgt, (void *)c->mlp_mask,
                  (void *)c->squeue, c->squeue_buf})
    if (p) cudaFree(p);
  void *bufs[] = {c->nu0,  c->S0,     c->El,    c->gair,   c->gself,  c->ncoll,
                  c->delta, c->lmass, c->lweight, c->rec64, c->rec32, c->core_rng, c->ckey, c->ckey32, c->tile_lo, c->tile_hi,
                  c->stats, c->kappa, c->sort_a, c->sort_b, c->pinv,  c->coef_dev,
                  c->mean_dev, c->tmp, c->kd_fold, c->kd_part, c->kd_done, c->tr_pairs, c->tr_bins};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (c->stats_host) cudaFreeHost(c->stats_host);
  if (c->cond_dev) cudaFree(c->cond_dev);
  if (c->cstats) cudaFree(c->cstats);
  if (c->cond_order) cudaFree(c->cond_order);
  if (c->cond_host) cudaFreeHost(c->cond_host);
  if (c->cstats_host) cudaFreeHost(c->cstats_host);
  if (c->cond_ev) cudaEventDestroy(c->cond_ev);
  for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->kcore) cudaFree(c->kcore);
  if (c->core_blk) cudaFree(c->core_blk);
  for (int st = 0; st < HELK_NSTAGES; ++st)
    for (cudaEvent_t e : c->ev[st]) cudaEventDestroy(e);
  if (cur >= 0) cudaSetDevice(cur);
  delete c;
}

const char *helk_last_error(const helk_ctx *c) { return c ? c->err.c_str() : "null context"; }

helk_status helk_set_stream(helk_ctx *c, void *stream) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return HELK_OK;
}

helk_status helk_sync(helk_ctx *c) {
  if (!c) return HELK_ERR_INVALID_ARG;
  HELK_TRY(bind_device(c));
  HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "stream synchronize"));
  HELK_TRY(cuda_check(c, cudaMemcpy(c->stats_host, c->stats, sizeof(DevStats), cudaMemcpyDeviceToHost),
                      "read status"));
  const int flags = c->stats_host->err_flags;
  if (flags) {
    // report once, then clear: the context stays usable
    HELK_TRY(cuda_check(c, cudaMemset(&c->stats->err_flags, 0, sizeof(int)), "clear status"));
    if (flags & ERRF_TIMEOUT) return set_err(c, HELK_ERR_TIMEOUT, "a kernel's bounded wait gave up");
    if (flags & ERRF_F32_RANGE)
      return set_err(c, HELK_ERR_UNSUPPORTED,
                     "FP32 form: a line's core reaches beyond 2^23 grid points of its centre "
                     "(Doppler width above ~7e5 grid steps); use the FP64 form");
  }
  return HELK_OK;
}

helk_status helk_lines_upload(helk_ctx *c, const helk_lines *L, int64_t n, int32_t on_device) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (!L || n < 0 || n > INT32_MAX - 1)
    return set_err(c, HELK_ERR_INVALID_ARG, "lines_upload: null lines or n out of range");
  if (n > 0 && (!L->nu0 || !L->S0 || !L->gamma_air))
    return set_err(c, HELK_ERR_INVALID_ARG, "lines_upload: nu0, S0 and gamma_air are required");
  HELK_TRY(bind_device(c));
  const int64_t bytes = (n > 0 ? n : 1) * 8;
  double **dst[9] = {&c->nu0, &c->S0, &c->El, &c->gair, &c->gself, &c->ncoll, &c->delta, &c->lmass,
                     &c->lweight};
  const double *src[9] = {L->nu0, L->S0, L->E_lower, L->gamma_air, L->gamma_self, L->n_coll, L->delta,
                          L->mass, L->weight};
  if (bytes > c->lines_cap) {
    HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "lines_upload"));
    for (auto d : dst)
      if (*d) {
        cudaFree(*d);
        *d = nullptr;
      }
    c->lines_cap = 0;
    for (auto d : dst) HELK_TRY(cuda_check(c, cudaMalloc((void **)d, (size_t)bytes), "lines_upload alloc"));
    c->lines_cap = bytes;
  }
  c->nlines = 0;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int f = 0; f < 9; ++f)
    if (src[f] && n > 0)
      HELK_TRY(cuda_check(c, cudaMemcpyAsync(*dst[f], src[f], (size_t)(n * 8), kind, c->stream),
                          "lines_upload copy"));
  c->has_E = L->E_lower != nullptr;
  c->has_gself = L->gamma_self != nullptr;
  c->has_ncoll = L->n_coll != nullptr;
  c->has_delta = L->delta != nullptr;
  c->has_mass = L->mass != nullptr;
  c->has_weight = L->weight != nullptr;
  HELK_TRY(cuda_check(c, cudaMemsetAsync(&c->stats->bad_lines, 0, 2 * sizeof(int), c->stream),
                      "lines_upload"));
  HELK_TRY(cuda_check(c, launch_validate_lines(c, n), "validate lines"));
  HELK_TRY(cuda_check(c, cudaMemcpyAsync(c->stats_host, c->stats, sizeof(DevStats),
                                         cudaMemcpyDeviceToHost, c->stream),
                      "lines_upload"));
  HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "lines_upload"));
  if (c->stats_host->bad_lines)
    return set_err(c, HELK_ERR_INVALID_ARG,
                   "lines_upload: " + std::to_string(c->stats_host->bad_lines) +
                       " lines with non-finite or negative values");
  if (c->stats_host->unsorted) {
    HELK_TRY(cuda_check(c, launch_sort_lines(c, n), "sort lines"));
    HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sort lines"));
  }
  c->nlines = n;
  c->have_opacity = false;
  return HELK_OK;
}

static helk_status check_condition(helk_ctx *c, double T, double P, double mass, const helk_cutoff *cut,
                                   const helk_grid *g, const helk_opts &o) {
  if (!cut || !g) return set_err(c, HELK_ERR_INVALID_ARG, "null cutoff or grid");
  if (!(is_fin(T) && T > 0.0)) return set_err(c, HELK_ERR_INVALID_ARG, "T must be finite and > 0");
  if (!(is_fin(P) && P >= 0.0)) return set_err(c, HELK_ERR_INVALID_ARG, "P must be finite and >= 0");
  if (!(is_fin(mass) && mass > 0.0)) return set_err(c, HELK_ERR_INVALID_ARG, "mass must be > 0");
  if (!(is_fin(g->nu_min) && is_fin(g->dnu) && g->dnu > 0.0))
    return set_err(c, HELK_ERR_INVALID_ARG, "grid: nu_min finite, dnu > 0 required");
  if (g->n <= 0 || g->n > INT32_MAX - 4096)
    return set_err(c, HELK_ERR_INVALID_ARG, "grid: n must be in [1, 2^31 - 4097]");
  if (cut->kind < HELK_CUT_ABS || cut->kind > HELK_CUT_NONE)
    return set_err(c, HELK_ERR_INVALID_ARG, "cutoff: unknown kind");
  if (cut->kind != HELK_CUT_NONE && !(is_fin(cut->value) && cut->value >= 0.0))
    return set_err(c, HELK_ERR_INVALID_ARG, "cutoff: value must be finite and >= 0");
  if (cut->kind == HELK_CUT_LORENTZ && !(is_fin(cut->cap) && cut->cap >= 0.0))
    return set_err(c, HELK_ERR_INVALID_ARG, "cutoff: cap must be finite and >= 0");
  if (o.precision != HELK_PREC_F64 && o.precision != HELK_PREC_F32_KAHAN)
    return set_err(c, HELK_ERR_INVALID_ARG, "opts: unknown precision");
  if (!is_fin(o.weight) || !(is_fin(o.q_ratio) && o.q_ratio > 0.0))
    return set_err(c, HELK_ERR_INVALID_ARG, "opts: weight finite and q_ratio > 0 required");
  if (o.surrogate && o.precision != HELK_PREC_F32_KAHAN)
    return set_err(c, HELK_ERR_INVALID_ARG, "opts: the surrogate is used by the FP32 form only");
  if (o.surrogate && !c->mlp_mask)
    return set_err(c, HELK_ERR_STATE, "opts: surrogate requested but no network has been validated");
  return HELK_OK;
}

static helk_opts default_opts() {
  helk_opts o;
  o.precision = HELK_PREC_F64;
  o.accumulate = 0;
  o.weight = 1.0;
  o.q_ratio = 1.0;
  o.count_regions = 0;
  o.surrogate = 0;
  return o;
}

static helk_status ensure_tiles(helk_ctx *c, int64_t ntiles) {
  if (ntiles <= c->tile_cap) return HELK_OK;
  if (c->tile_lo) cudaFree(c->tile_lo);
  if (c->tile_hi) cudaFree(c->tile_hi);
  c->tile_lo = c->tile_hi = nullptr;
  c->tile_cap = 0;
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->tile_lo, (size_t)ntiles * 4), "tile map"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->tile_hi, (size_t)ntiles * 4), "tile map"));
  c->tile_cap = ntiles;
  return HELK_OK;
}

// Room for n_cond conditions: parameter staging, per-condition statistics,
// the condition order.
static helk_status ensure_conds(helk_ctx *c, int n_cond) {
  if (n_cond <= c->cond_cap) return HELK_OK;
  HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "conditions"));
  if (c->cond_dev) cudaFree(c->cond_dev);
  if (c->cstats) cudaFree(c->cstats);
  if (c->cond_order) cudaFree(c->cond_order);
  if (c->cond_host) cudaFreeHost(c->cond_host);
  if (c->cstats_host) cudaFreeHost(c->cstats_host);
  c->cond_dev = nullptr;
  c->cstats = nullptr;
  c->cond_order = nullptr;
  c->cond_host = nullptr;
  c->cstats_host = nullptr;
  c->cond_cap = 0;
  const int cap = std::max(n_cond, 8);
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->cond_dev, cap * sizeof(CondArgs)), "conditions"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->cstats, cap * sizeof(CondStats)), "conditions"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->cond_order, cap * sizeof(int)), "conditions"));
  HELK_TRY(cuda_check(c, cudaMallocHost((void **)&c->cond_host, cap * sizeof(CondArgs)), "conditions"));
  HELK_TRY(cuda_check(c, cudaMallocHost((void **)&c->cstats_host, cap * sizeof(CondStats)), "conditions"));
  c->cond_cap = cap;
  return HELK_OK;
}

// Buffers for n_cond conditions of the current line list and tile shape.
static helk_status ensure_call_buffers(helk_ctx *c, int n_cond, const helk_opts &o, int64_t ntiles,
                                       int64_t ngrid) {
  const int64_t nl = std::max<int64_t>(c->nlines, 1) * n_cond;
  HELK_TRY(ensure_conds(c, n_cond));
  HELK_TRY(ensure_buf(c, (void **)&c->rec64, &c->rec_cap, nl * (int64_t)sizeof(LineRec64), "line records"));
  HELK_TRY(ensure_buf(c, (void **)&c->ckey, &c->ckey_cap, std::max<int64_t>(c->nlines, 1) * 8, "line keys"));
  if (o.precision == HELK_PREC_F32_KAHAN) {
    HELK_TRY(ensure_buf(c, (void **)&c->rec32, &c->rec32_cap, nl * (int64_t)sizeof(LineRec32),
                        "FP32 line records"));
    HELK_TRY(ensure_buf(c, (void **)&c->core_rng, &c->core_cap, nl * (int64_t)sizeof(int2), "line cores"));
    HELK_TRY(ensure_buf(c, (void **)&c->ckey32, &c->ckey32_cap, std::max<int64_t>(c->nlines, 1) * 4,
                        "line keys"));
    HELK_TRY(ensure_buf(c, (void **)&c->kcore, &c->kcore_cap, ngrid * n_cond * 4, "core sums"));
    HELK_TRY(ensure_buf(c, (void **)&c->core_blk, &c->core_blk_cap, (int64_t)core_blocks(ngrid) * n_cond * 4,
                        "core reach"));
    if (!c->side_stream)
      HELK_TRY(cuda_check(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking), "core stream"));
    if (!c->fork_ev)
      HELK_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming), "core stream"));
    if (!c->join_ev)
      HELK_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming), "core stream"));
  }
  HELK_TRY(ensure_tiles(c, ntiles * n_cond));
  if (o.surrogate && !c->squeue) {
    // routed-evaluation queue: 2^24 entries (entries beyond it fall back to
    // Algorithm 916 in the Voigt kernel)
    const int64_t cap = (int64_t)1 << 24;
    HELK_TRY(cuda_check(c, cudaMalloc(&c->squeue_buf, (size_t)cap * 20), "surrogate queue"));
    HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->squeue, sizeof(SurrQueue)), "surrogate queue"));
    SurrQueue q;
    q.count = 0;
    q.cap = (unsigned)cap;
    char *b = (char *)c->squeue_buf;
    q.idx = (int32_t *)b;
    q.cond = (int32_t *)(b + cap * 4);
    q.w = (float *)(b + cap * 8);
    q.x = (float *)(b + cap * 12);
    q.y = (float *)(b + cap * 16);
    q.mask = c->mlp_mask;
    q.nx = c->mlp_mask_nx;
    q.ny = c->mlp_mask_ny;
    HELK_TRY(cuda_check(c, cudaMemcpy(c->squeue, &q, sizeof q, cudaMemcpyHostToDevice), "surrogate queue"));
    c->squeue_cap = cap;
  }
  return HELK_OK;
}

// Statistics reset and line preparation (and the FP32 records) of n_cond
// conditions: single != NULL passes the one condition by value, otherwise
// they are read from c->cond_dev.
static helk_status prepare_lines(helk_ctx *c, int n_cond, const CondArgs *single, double mass,
                                 const helk_cutoff *cut, const helk_grid *g, const helk_opts &o) {
  HELK_TRY(cuda_check(c, cudaMemsetAsync(c->cstats, 0, n_cond * sizeof(CondStats), c->stream), "stats"));
  for (int k = 0; k < n_cond; ++k)
    HELK_TRY(cuda_check(c, cudaMemsetAsync(&c->cstats[k].wmax, 0xFF, sizeof(long long), c->stream), "stats"));
  if (c->nlines > 0) {
    HELK_TRY(cuda_check(c, launch_lineprep(c, n_cond, single, mass, *cut, *g, o.precision != HELK_PREC_F32_KAHAN),
                        "lineprep"));
    if (o.precision == HELK_PREC_F32_KAHAN) {
      HELK_TRY(cuda_check(c, cudaMemsetAsync(c->core_blk, 0, (size_t)core_blocks(g->n) * n_cond * 4, c->stream),
                          "pack32"));
      HELK_TRY(cuda_check(c, launch_pack32(c, n_cond, *g), "pack32"));
    }
  }
  return HELK_OK;
}

// Points per CTA tile of a shape code returned by voigt_shape or the
// candidates (codes that always decode; 0 would mean a logic error, which
// the callers report).
static int shape_points(int precision, int shape) {
  int p = 0;
  return voigt_shape_info(precision, shape, &p, nullptr, nullptr) ? p : 0;
}

// Tile map, condition order and the persistent Voigt kernel (for the FP32
// form with its Algorithm 916 cores).  `shape`: the Voigt kernel's shape
// code; `tile`: its points per CTA tile.
static helk_status run_voigt(helk_ctx *c, int n_cond, const helk_grid *g, const helk_opts &o, double *kappa,
                             int shape, int tile, int64_t ntiles) {
  HELK_TRY(cuda_check(c, launch_tilemap(c, n_cond, *g, tile, ntiles), "tilemap"));
  HELK_TRY(cuda_check(c, launch_cond_order(c, n_cond), "condition order"));
  HELK_TRY(cuda_check(c, cudaMemsetAsync(&c->stats->tile_counter, 0, sizeof(unsigned int), c->stream),
                      "voigt"));
  if (o.surrogate)
    HELK_TRY(cuda_check(c, cudaMemsetAsync(&c->squeue->count, 0, sizeof(unsigned long long), c->stream), "voigt"));
  if (o.precision == HELK_PREC_F32_KAHAN) {
    // The Algorithm 916 cores run on the side stream beside the main kernel
    // (whose CTAs are issued first and leave registers and warp slots on every
    // SM), into their own buffer; their sums are added once both are done.
    HELK_TRY(cuda_check(c, cudaEventRecord(c->fork_ev, c->stream), "voigt"));
    HELK_TRY(cuda_check(c, launch_voigt(c, n_cond, *g, o, kappa, shape, ntiles), "voigt"));
    HELK_TRY(cuda_check(c, cudaStreamWaitEvent(c->side_stream, c->fork_ev, 0), "voigt cores"));
    HELK_TRY(cuda_check(c, launch_voigt_core(c, n_cond, *g, o), "voigt cores"));
    HELK_TRY(cuda_check(c, cudaEventRecord(c->join_ev, c->side_stream), "voigt cores"));
    HELK_TRY(cuda_check(c, cudaStreamWaitEvent(c->stream, c->join_ev, 0), "voigt cores"));
    HELK_TRY(cuda_check(c, launch_core_add(c, n_cond, *g, o, kappa), "voigt cores"));
  } else {
    HELK_TRY(cuda_check(c, launch_voigt(c, n_cond, *g, o, kappa, shape, ntiles), "voigt"));
  }
  if (o.surrogate) HELK_TRY(cuda_check(c, launch_mlp_queue(c, n_cond, g->n, o.weight, kappa), "surrogate"));
  return HELK_OK;
}

helk_status helk_opacity(helk_ctx *c, double T, double P, double mass, const helk_cutoff *cut,
                         const helk_grid *g, const helk_opts *opts, double *kappa_out) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  const helk_opts o = opts ? *opts : default_opts();
  HELK_TRY(check_condition(c, T, P, mass, cut, g, o));
  if (!c->nu0) return set_err(c, HELK_ERR_STATE, "opacity: no line list uploaded");
  HELK_TRY(bind_device(c));
  double *kappa = kappa_out;
  if (!kappa) {
    HELK_TRY(ensure_buf(c, (void **)&c->kappa, &c->kappa_cap, g->n * 8, "opacity buffer"));
    kappa = c->kappa;
  }
  const int shape = voigt_shape(c, o.precision, o.count_regions, g->n);
  const int tile = shape_points(o.precision, shape);
  if (tile <= 0) return set_err(c, HELK_ERR_STATE, "opacity: no kernel shape");
  const int64_t ntiles = (g->n + tile - 1) / tile;
  HELK_TRY(ensure_call_buffers(c, 1, o, ntiles, g->n));
  const CondArgs one{T, P, o.q_ratio, 0.0};
  stage_begin(c, HELK_STAGE_LINEPREP);
  HELK_TRY(prepare_lines(c, 1, &one, mass, cut, g, o));
  stage_end(c, HELK_STAGE_LINEPREP);
  if (c->nlines > 0) {
    stage_begin(c, HELK_STAGE_VOIGT);
    HELK_TRY(run_voigt(c, 1, g, o, kappa, shape, tile, ntiles));
    stage_end(c, HELK_STAGE_VOIGT);
  } else if (!o.accumulate) {
    HELK_TRY(cuda_check(c, cudaMemsetAsync(kappa, 0, (size_t)g->n * 8, c->stream), "opacity"));
  }
  c->last_n = g->n;
  c->last_ncond = 1;
  c->have_opacity = (kappa == c->kappa);
  c->last_counted_regions = o.count_regions != 0;
  return HELK_OK;
}

helk_status helk_autotune(helk_ctx *c, double T, double P, double mass, const helk_cutoff *cut,
                          const helk_grid *g, const helk_opts *opts, int32_t *tile_out) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  helk_opts o = opts ? *opts : default_opts();
  o.count_regions = 0;
  o.accumulate = 0;
  HELK_TRY(check_condition(c, T, P, mass, cut, g, o));
  if (!c->nu0 || c->nlines <= 0) return set_err(c, HELK_ERR_STATE, "autotune: no line list uploaded");
  HELK_TRY(bind_device(c));
  HELK_TRY(ensure_buf(c, (void **)&c->kappa, &c->kappa_cap, g->n * 8, "opacity buffer"));
  const int prec = o.precision == HELK_PREC_F32_KAHAN ? 1 : 0;
  c->tuned_tile[prec] = 0;  // time the candidates, not the previous choice
  int cand[32];
  const int ncand = voigt_shape_candidates(o.precision, cand, 32);
  int64_t max_tiles = 0;
  for (int i = 0; i < ncand; ++i) {
    const int pts = std::max(1, shape_points(o.precision, cand[i]));
    max_tiles = std::max(max_tiles, (g->n + pts - 1) / pts);
  }
  HELK_TRY(ensure_call_buffers(c, 1, o, max_tiles, g->n));
  const CondArgs one{T, P, o.q_ratio, 0.0};
  HELK_TRY(prepare_lines(c, 1, &one, mass, cut, g, o));
  cudaEvent_t e0, e1;
  HELK_TRY(cuda_check(c, cudaEventCreate(&e0), "autotune"));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_check(c, cudaErrorUnknown, "autotune");
  }
  double best_ms = 1e300;
  int best = cand[0];
  helk_status st = HELK_OK;
  for (int i = 0; i < ncand && st == HELK_OK; ++i) {
    const int pts = std::max(1, shape_points(o.precision, cand[i]));
    const int64_t ntiles = (g->n + pts - 1) / pts;
    st = run_voigt(c, 1, g, o, c->kappa, cand[i], pts, ntiles);  // warm-up
    float ms = 0.f;
    const int reps = 3;
    if (st == HELK_OK) st = cuda_check(c, cudaEventRecord(e0, c->stream), "autotune");
    for (int r = 0; r < reps && st == HELK_OK; ++r) st = run_voigt(c, 1, g, o, c->kappa, cand[i], pts, ntiles);
    if (st == HELK_OK) st = cuda_check(c, cudaEventRecord(e1, c->stream), "autotune");
    if (st == HELK_OK) st = cuda_check(c, cudaEventSynchronize(e1), "autotune");
    if (st == HELK_OK) st = cuda_check(c, cudaEventElapsedTime(&ms, e0, e1), "autotune");
    if (st == HELK_OK && ms / reps < best_ms) {
      best_ms = ms / reps;
      best = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HELK_TRY(st);
  HELK_TRY(helk_sync(c));
  c->tuned_tile[prec] = best;
  c->tuned_n[prec] = g->n;
  c->have_opacity = false;
  if (tile_out) *tile_out = best;
  return HELK_OK;
}

// ---------------------------------------------------------------- batch --

// Many (T, P) conditions in one persistent Voigt launch; the whole sequence
// (condition upload from pinned staging, statistics reset, line preparation,
// FP32 records, tile maps, condition order, Voigt kernel) is captured once
// into a CUDA graph per call shape and replayed.
static std::string batch_key(const helk_ctx *c, int n_cond, double mass, const helk_cutoff *cut,
                             const helk_grid *g, const helk_opts &o, const double *kappa, int shape) {
  char b[512];
  snprintf(b, sizeof b, "%d|%lld|%p|%a|%d|%a|%a|%a|%a|%lld|%d|%d|%a|%d|%d|%p|%d|%p|%p|%p|%p|%p|%p", n_cond,
           (long long)c->nlines, (const void *)c->nu0, mass, cut->kind, cut->value, cut->cap, g->nu_min,
           g->dnu, (long long)g->n, o.precision, o.accumulate, o.weight, o.count_regions, o.surrogate,
           (const void *)kappa, shape, (const void *)c->rec64, (const void *)c->rec32,
           (const void *)c->tile_lo, (const void *)c->cstats, (const void *)c->squeue, (const void *)c->kcore);
  // the line fields present (absent ones are passed to line preparation as
  // null pointers) and the per-condition arrays of the chunk
  char b2[192];
  snprintf(b2, sizeof b2, "|%d%d%d%d%d%d|%p|%p|%p|%p", c->has_E, c->has_gself, c->has_ncoll, c->has_delta,
           c->has_mass, c->has_weight, (const void *)c->cond_host, (const void *)c->cond_dev,
           (const void *)c->cond_order, (const void *)c->core_rng);
  char b3[64];
  snprintf(b3, sizeof b3, "|%p", (const void *)c->core_blk);
  return std::string(b) + b2 + b3;
}

// The per-condition arrays as seen by a chunk of a batch: offset by the
// chunk's first condition for the lifetime of the view.
struct CondView {
  helk_ctx *c;
  int k0;
  CondView(helk_ctx *ctx, int first) : c(ctx), k0(first) {
    c->cond_host += k0;
    c->cond_dev += k0;
    c->cstats += k0;
    c->cond_order += k0;
  }
  ~CondView() {
    c->cond_host -= k0;
    c->cond_dev -= k0;
    c->cstats -= k0;
    c->cond_order -= k0;
  }
  CondView(const CondView &) = delete;
  CondView &operator=(const CondView &) = delete;
};

static cudaGraphExec_t find_graph(helk_ctx *c, const std::string &key) {
  for (auto &kv : c->graphs)
    if (kv.first == key) return kv.second;
  return nullptr;
}

// Keeps the last MAX_GRAPHS captured graphs (a graph still running when it
// is dropped is freed when it completes).
static void keep_graph(helk_ctx *c, const std::string &key, cudaGraphExec_t gx) {
  constexpr size_t MAX_GRAPHS = 16;
  if (c->graphs.size() >= MAX_GRAPHS) {
    cudaGraphExecDestroy(c->graphs.front().second);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.emplace_back(key, gx);
}

helk_status helk_opacity_batch(helk_ctx *c, int32_t n_cond, const double *T, const double *P,
                               const double *q_ratio, double mass, const helk_cutoff *cut,
                               const helk_grid *g, const helk_opts *opts, double *kappa_out) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (n_cond < 1 || !T || !P) return set_err(c, HELK_ERR_INVALID_ARG, "opacity_batch: need n_cond >= 1, T, P");
  const helk_opts o = opts ? *opts : default_opts();
  for (int k = 0; k < n_cond; ++k) {
    helk_opts ok = o;
    if (q_ratio) ok.q_ratio = q_ratio[k];
    HELK_TRY(check_condition(c, T[k], P[k], mass, cut, g, ok));
  }
  if ((int64_t)n_cond * g->n > ((int64_t)1 << 40))
    return set_err(c, HELK_ERR_INVALID_ARG, "opacity_batch: n_cond * grid size too large");
  if (!c->nu0) return set_err(c, HELK_ERR_STATE, "opacity_batch: no line list uploaded");
  HELK_TRY(bind_device(c));
  double *kappa = kappa_out;
  if (!kappa) {
    HELK_TRY(ensure_buf(c, (void **)&c->kappa, &c->kappa_cap, (int64_t)n_cond * g->n * 8, "opacity buffer"));
    kappa = c->kappa;
  }
  if (c->nlines <= 0) {
    if (!o.accumulate)
      HELK_TRY(cuda_check(c, cudaMemsetAsync(kappa, 0, (size_t)n_cond * g->n * 8, c->stream), "opacity"));
    c->last_n = g->n * n_cond;
    c->last_ncond = n_cond;
    c->have_opacity = (kappa == c->kappa);
    return HELK_OK;
  }
  const int shape = voigt_shape(c, o.precision, o.count_regions, g->n);
  const int tile = shape_points(o.precision, shape);
  if (tile <= 0) return set_err(c, HELK_ERR_STATE, "opacity: no kernel shape");
  const int64_t ntiles = (g->n + tile - 1) / tile;
  // Conditions run in the fewest equal chunks whose line records fit the
  // record budget (one chunk unless the list is very long), each chunk one
  // captured graph; the chunks share the record, tile-map and core buffers
  // and follow each other on the stream.
  const int64_t rec_line =
      (int64_t)sizeof(LineRec64) +
      (o.precision == HELK_PREC_F32_KAHAN ? (int64_t)(sizeof(LineRec32) + sizeof(int2)) : 0);
  const int64_t per_cond = std::max<int64_t>(c->nlines, 1) * rec_line;
  const int gmax = (int)std::max<int64_t>(1, std::min<int64_t>(n_cond, c->batch_budget / per_cond));
  const int nchunk = (n_cond + gmax - 1) / gmax;
  const int chunk = (n_cond + nchunk - 1) / nchunk;
  HELK_TRY(ensure_conds(c, n_cond));
  HELK_TRY(ensure_call_buffers(c, chunk, o, ntiles, g->n));
  if (!c->cap_stream)
    HELK_TRY(cuda_check(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "graph stream"));
  if (!c->cond_ev) HELK_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->cond_ev, cudaEventDisableTiming), "graph"));
  // the previous batch must have read the staging buffer before it changes
  HELK_TRY(cuda_check(c, cudaEventSynchronize(c->cond_ev), "opacity_batch"));
  for (int k = 0; k < n_cond; ++k) c->cond_host[k] = CondArgs{T[k], P[k], q_ratio ? q_ratio[k] : o.q_ratio, 0.0};
  stage_begin(c, HELK_STAGE_VOIGT);
  for (int j = 0; j < nchunk; ++j) {
    const int k0 = j * chunk, nk = std::min(chunk, n_cond - k0);
    double *kap = kappa + (int64_t)k0 * g->n;
    cudaGraphExec_t gx = nullptr;
    {
      // the chunk's view of the per-condition arrays (staging, parameters,
      // statistics, order): offset by its first condition, restored after
      const CondView view(c, k0);
      const std::string key = batch_key(c, nk, mass, cut, g, o, kap, shape);
      gx = find_graph(c, key);
      if (!gx) {
        cudaStream_t user = c->stream;
        c->stream = c->cap_stream;
        cudaGraph_t graph = nullptr;
        helk_status st = cuda_check(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal),
                                    "graph capture");
        if (st == HELK_OK) {
          st = cuda_check(c, cudaMemcpyAsync(c->cond_dev, c->cond_host, nk * sizeof(CondArgs),
                                             cudaMemcpyHostToDevice, c->stream),
                          "graph capture");
          if (st == HELK_OK) st = prepare_lines(c, nk, nullptr, mass, cut, g, o);
          if (st == HELK_OK) st = run_voigt(c, nk, g, o, kap, shape, tile, ntiles);
          const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
          if (st == HELK_OK) st = cuda_check(c, e, "graph capture");
        }
        c->stream = user;
        if (st == HELK_OK) st = cuda_check(c, cudaGraphInstantiate(&gx, graph, 0), "graph instantiate");
        if (graph) cudaGraphDestroy(graph);
        if (st != HELK_OK) {
          cudaGetLastError();
          return st;
        }
        keep_graph(c, key, gx);
      }
    }
    HELK_TRY(cuda_check(c, cudaGraphLaunch(gx, c->stream), "graph launch"));
  }
  stage_end(c, HELK_STAGE_VOIGT);
  HELK_TRY(cuda_check(c, cudaEventRecord(c->cond_ev, c->stream), "opacity_batch"));
  c->last_n = g->n * n_cond;
  c->last_ncond = n_cond;
  c->have_opacity = (kappa == c->kappa);
  c->last_counted_regions = o.count_regions != 0;
  return HELK_OK;
}

helk_status helk_set_batch_budget(helk_ctx *c, int64_t bytes) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (bytes < 0) return set_err(c, HELK_ERR_INVALID_ARG, "set_batch_budget: bytes must be >= 0");
  c->batch_budget = bytes > 0 ? bytes : HELK_DEFAULT_BATCH_BUDGET;
  return HELK_OK;
}

helk_status helk_opacity_batch_stats(helk_ctx *c, int32_t n_cond, int64_t *n_evals, int64_t *region_counts) {
  if (!c || n_cond < 1) return HELK_ERR_INVALID_ARG;
  if (n_cond > c->last_ncond) return set_err(c, HELK_ERR_STATE, "batch_stats: more conditions than the last call");
  HELK_TRY(helk_sync(c));
  HELK_TRY(cuda_check(c, cudaMemcpy(c->cstats_host, c->cstats, n_cond * sizeof(CondStats), cudaMemcpyDeviceToHost),
                      "batch_stats"));
  if (region_counts && !c->last_counted_regions)
    return set_err(c, HELK_ERR_STATE, "batch_stats: last call ran without count_regions");
  for (int k = 0; k < n_cond; ++k) {
    if (n_evals) n_evals[k] = (int64_t)c->cstats_host[k].evals;
    if (region_counts)
      for (int r = 0; r < 4; ++r) region_counts[4 * k + r] = (int64_t)c->cstats_host[k].region[r];
  }
  return HELK_OK;
}

helk_status helk_opacity_stats(helk_ctx *c, int64_t *n_evals, int64_t *region_counts) {
  if (!c) return HELK_ERR_INVALID_ARG;
  if (c->last_ncond < 1) return set_err(c, HELK_ERR_STATE, "opacity_stats: no opacity computed yet");
  return helk_opacity_batch_stats(c, 1, n_evals, region_counts);
}

helk_status helk_kdist(helk_ctx *c, const double *kappa, int64_t n, int32_t nbins, int32_t ncheb,
                       double kappa_floor, double *coeffs, double *mean, int32_t out_on_host,
                       double *kg_out) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (n <= 0 || n > INT32_MAX || nbins <= 0 || n % nbins)
    return set_err(c, HELK_ERR_INVALID_ARG, "kdist: n must be a positive multiple of nbins");
  const int64_t nb = n / nbins;
  if (ncheb < 1 || ncheb > 32 || ncheb > nb)
    return set_err(c, HELK_ERR_INVALID_ARG, "kdist: need 1 <= ncheb <= min(32, n/nbins)");
  if (!(is_fin(kappa_floor) && kappa_floor > 0.0))
    return set_err(c, HELK_ERR_INVALID_ARG, "kdist: kappa_floor must be finite and > 0");
  if (!coeffs) return set_err(c, HELK_ERR_INVALID_ARG, "kdist: coeffs is required");
  if (!kappa) {
    if (!c->have_opacity || c->last_n != n)
      return set_err(c, HELK_ERR_STATE, "kdist: no context opacity of this size");
    kappa = c->kappa;
  }
  HELK_TRY(bind_device(c));
  if (c->pinv_nb != nb || c->pinv_ncheb != ncheb || !c->pinv) {
    HELK_TRY(ensure_buf(c, (void **)&c->pinv, &c->pinv_cap, pinv_bytes(nb, ncheb), "kdist pseudo-inverse"));
    HELK_TRY(ensure_buf(c, &c->tmp, &c->tmp_cap, pinv_work_doubles(nb, ncheb) * 8, "kdist pseudo-inverse"));
    stage_begin(c, HELK_STAGE_SETUP);
    HELK_TRY(cuda_check(c, launch_pinv(c, nb, ncheb, (double *)c->tmp), "kdist pseudo-inverse"));
    stage_end(c, HELK_STAGE_SETUP);
    c->pinv_nb = nb;
    c->pinv_ncheb = ncheb;
  }
  {  // the global sort buffers: the bins too large for shared memory, and the
     // radix passes of a bin whose bucket sort gives up
    if (n * 8 > c->sort_cap) {
      HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "kdist"));
      if (c->sort_a) cudaFree(c->sort_a);
      if (c->sort_b) cudaFree(c->sort_b);
      c->sort_a = c->sort_b = nullptr;
      c->sort_cap = 0;
      HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->sort_a, (size_t)n * 8), "kdist scratch"));
      HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->sort_b, (size_t)n * 8), "kdist scratch"));
      c->sort_cap = n * 8;
    }
  }
  HELK_TRY(ensure_buf(c, &c->kd_fold, &c->kd_fold_cap, kdist_fold_bytes(n, nbins), "kdist scratch"));
  HELK_TRY(ensure_buf(c, &c->kd_part, &c->kd_part_cap, kdist_part_bytes(c, n, nbins), "kdist scratch"));
  if (kdist_done_bytes(nbins) > c->kd_done_cap) {
    HELK_TRY(ensure_buf(c, &c->kd_done, &c->kd_done_cap, kdist_done_bytes(nbins), "kdist scratch"));
    HELK_TRY(cuda_check(c, cudaMemsetAsync(c->kd_done, 0, (size_t)c->kd_done_cap, c->stream), "kdist scratch"));
  }
  double *cdst = coeffs, *mdst = mean;
  if (out_on_host) {
    HELK_TRY(ensure_buf(c, (void **)&c->coef_dev, &c->coef_cap, (int64_t)nbins * ncheb * 8, "kdist out"));
    HELK_TRY(ensure_buf(c, (void **)&c->mean_dev, &c->mean_cap, (int64_t)nbins * 8, "kdist out"));
    cdst = c->coef_dev;
    mdst = c->mean_dev;
  }
  stage_begin(c, HELK_STAGE_KDIST);
  HELK_TRY(cuda_check(c, launch_kdist_bins(c, kappa, n, nbins, ncheb, kappa_floor, cdst, mdst, kg_out),
                      "kdist"));
  stage_end(c, HELK_STAGE_KDIST);
  if (out_on_host) {
    HELK_TRY(cuda_check(c, cudaMemcpyAsync(coeffs, cdst, (size_t)nbins * ncheb * 8, cudaMemcpyDeviceToHost,
                                           c->stream),
                        "kdist copy"));
    if (mean)
      HELK_TRY(cuda_check(c, cudaMemcpyAsync(mean, mdst, (size_t)nbins * 8, cudaMemcpyDeviceToHost, c->stream),
                          "kdist copy"));
    HELK_TRY(helk_sync(c));
  }
  return HELK_OK;
}

helk_status helk_transmission(helk_ctx *c, int32_t nbins, int64_t nb, const double *sorted,
                              const double *coeffs, int32_t ncheb, int32_t ng, int32_t nm,
                              const double *m, double *direct, double *fit) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (nbins < 1 || nm < 1 || !m) return set_err(c, HELK_ERR_INVALID_ARG, "transmission: nbins, nm >= 1 and m required");
  if (sorted && (nb < 1 || !direct)) return set_err(c, HELK_ERR_INVALID_ARG, "transmission: nb >= 1 and direct required");
  if (coeffs && (ncheb < 1 || ncheb > 32 || ng < 1 || ng > 16384 || !fit))
    return set_err(c, HELK_ERR_INVALID_ARG, "transmission: 1 <= ncheb <= 32, 1 <= ng <= 16384 and fit required");
  if (!sorted && !coeffs) return set_err(c, HELK_ERR_INVALID_ARG, "transmission: nothing to do");
  for (int i = 0; i < nm; ++i)
    if (!(is_fin(m[i]) && m[i] >= 0.0)) return set_err(c, HELK_ERR_INVALID_ARG, "transmission: m must be finite, >= 0");
  HELK_TRY(bind_device(c));
  HELK_TRY(ensure_buf(c, (void **)&c->mass_col, &c->mass_col_cap, (int64_t)nm * 8, "transmission"));
  if (sorted) {
    HELK_TRY(ensure_buf(c, &c->tr_pairs, &c->tr_pairs_cap, (int64_t)trans_pair_bytes(nbins, nb), "transmission"));
    HELK_TRY(ensure_buf(c, &c->tr_bins, &c->tr_bins_cap, (int64_t)trans_bin_bytes(nbins), "transmission"));
  }
  HELK_TRY(cuda_check(c, cudaMemcpyAsync(c->mass_col, m, (size_t)nm * 8, cudaMemcpyHostToDevice, c->stream),
                      "transmission"));
  HELK_TRY(cuda_check(c, launch_transmission(c, nbins, nb, sorted, coeffs, ncheb, ng, nm, c->mass_col, direct, fit),
                      "transmission"));
  // m is pageable host memory: the copy above has completed when it returned
  return HELK_OK;
}

// ------------------------------------------------------------ surrogate --
static helk_status ensure_mlp(helk_ctx *c) {
  if (c->mlp_p) return HELK_OK;
  const size_t nb = MLP_NPARAMS_H * sizeof(float);
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_p, nb), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_m, nb), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_v, nb), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_g, nb), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_loss, 64), "surrogate"));
  return HELK_OK;
}

static uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

helk_status helk_surrogate_init(helk_ctx *c, uint64_t seed) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  HELK_TRY(bind_device(c));
  HELK_TRY(ensure_mlp(c));
  // He-style normal initialisation (Box-Muller on SplitMix64 variates)
  std::vector<float> p(MLP_NPARAMS_H, 0.0f);
  uint64_t st = seed;
  auto normal = [&]() {
    const double u1 = ((splitmix64(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * PI * u2);
  };
  const int H = 64;
  for (int i = 0; i < 2 * H; ++i) p[i] = (float)(normal() * 1.0);                         // W1
  for (int i = 0; i < H * H; ++i) p[192 + i] = (float)(normal() * sqrt(2.0 / H));          // W2
  for (int i = 0; i < H * H; ++i) p[4352 + i] = (float)(normal() * sqrt(2.0 / H));         // W3
  for (int i = 0; i < H; ++i) p[8512 + i] = (float)(normal() * sqrt(1.0 / H) * 0.1);       // W4
  HELK_TRY(cuda_check(c, cudaMemcpy(c->mlp_p, p.data(), p.size() * 4, cudaMemcpyHostToDevice), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMemset(c->mlp_m, 0, p.size() * 4), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMemset(c->mlp_v, 0, p.size() * 4), "surrogate"));
  c->mlp_step = 0;
  return HELK_OK;
}

helk_status helk_surrogate_params(helk_ctx *c, float *get_host, const float *set_host) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  HELK_TRY(bind_device(c));
  HELK_TRY(ensure_mlp(c));
  HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "surrogate"));
  if (set_host) {
    HELK_TRY(cuda_check(c, cudaMemcpy(c->mlp_p, set_host, MLP_NPARAMS_H * 4, cudaMemcpyHostToDevice), "surrogate"));
    HELK_TRY(cuda_check(c, cudaMemset(c->mlp_m, 0, MLP_NPARAMS_H * 4), "surrogate"));
    HELK_TRY(cuda_check(c, cudaMemset(c->mlp_v, 0, MLP_NPARAMS_H * 4), "surrogate"));
    c->mlp_step = 0;
  }
  if (get_host)
    HELK_TRY(cuda_check(c, cudaMemcpy(get_host, c->mlp_p, MLP_NPARAMS_H * 4, cudaMemcpyDeviceToHost), "surrogate"));
  return HELK_OK;
}

static helk_status ensure_mlp_data(helk_ctx *c, int64_t n) {
  if (n <= c->mlp_data_cap) return HELK_OK;
  HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "surrogate data"));
  if (c->mlp_feat) cudaFree(c->mlp_feat);
  if (c->mlp_tgt) cudaFree(c->mlp_tgt);
  c->mlp_feat = c->mlp_tgt = nullptr;
  c->mlp_data_cap = 0;
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_feat, (size_t)n * 8), "surrogate data"));
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_tgt, (size_t)n * 4), "surrogate data"));
  c->mlp_data_cap = n;
  return HELK_OK;
}

helk_status helk_surrogate_samples(helk_ctx *c, int64_t n, uint64_t seed, float *feat, float *target,
                                   double *x, double *y) {
  if (!c || n < 1 || !feat || !target) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  HELK_TRY(bind_device(c));
  return cuda_check(c, launch_mlp_samples(c, n, seed, feat, target, x, y), "surrogate samples");
}

helk_status helk_surrogate_grad(helk_ctx *c, int64_t n, const float *feat, const float *target, float *grad_host,
                                double *loss_host) {
  if (!c || n < 1 || !feat || !target) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->mlp_p) return set_err(c, HELK_ERR_STATE, "surrogate: no network (call helk_surrogate_init)");
  HELK_TRY(bind_device(c));
  HELK_TRY(cuda_check(c, cudaMemsetAsync(c->mlp_g, 0, MLP_NPARAMS_H * 4, c->stream), "surrogate"));
  HELK_TRY(cuda_check(c, cudaMemsetAsync(c->mlp_loss, 0, 4, c->stream), "surrogate"));
  HELK_TRY(cuda_check(c, launch_mlp_train_step(c, c->mlp_p, feat, target, 0, n, c->mlp_g, c->mlp_loss), "surrogate"));
  HELK_TRY(helk_sync(c));
  if (grad_host)
    HELK_TRY(cuda_check(c, cudaMemcpy(grad_host, c->mlp_g, MLP_NPARAMS_H * 4, cudaMemcpyDeviceToHost), "surrogate"));
  if (loss_host) {
    float l = 0.f;
    HELK_TRY(cuda_check(c, cudaMemcpy(&l, c->mlp_loss, 4, cudaMemcpyDeviceToHost), "surrogate"));
    *loss_host = (double)l / (double)n;
  }
  return HELK_OK;
}

helk_status helk_surrogate_train(helk_ctx *c, int64_t n_samples, uint64_t seed, int32_t epochs, int32_t batch,
                                 double lr, double *final_loss) {
  if (!c || n_samples < 128 || epochs < 1 || batch < 128 || !(lr > 0.0)) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->mlp_p) return set_err(c, HELK_ERR_STATE, "surrogate: no network (call helk_surrogate_init)");
  HELK_TRY(bind_device(c));
  HELK_TRY(ensure_mlp_data(c, n_samples));
  HELK_TRY(cuda_check(c, launch_mlp_samples(c, n_samples, seed, c->mlp_feat, c->mlp_tgt, nullptr, nullptr),
                      "surrogate samples"));
  const int64_t steps_per_epoch = n_samples / batch;
  const int64_t total = steps_per_epoch * epochs;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    HELK_TRY(cuda_check(c, cudaMemsetAsync(c->mlp_loss, 0, 4, c->stream), "surrogate"));
    for (int64_t s = 0; s < steps_per_epoch; ++s) {
      // cosine decay of the learning rate to 1 % over the run
      const double prog = (double)(ep * steps_per_epoch + s) / (double)std::max<int64_t>(1, total);
      const float lr_s = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(PI * prog))));
      HELK_TRY(cuda_check(c, cudaMemsetAsync(c->mlp_g, 0, MLP_NPARAMS_H * 4, c->stream), "surrogate"));
      HELK_TRY(cuda_check(c, launch_mlp_train_step(c, c->mlp_p, c->mlp_feat, c->mlp_tgt, s * batch, batch,
                                                   c->mlp_g, c->mlp_loss),
                          "surrogate train"));
      HELK_TRY(cuda_check(c, launch_mlp_adam(c, c->mlp_p, c->mlp_m, c->mlp_v, c->mlp_g, lr_s, ++c->mlp_step),
                          "surrogate train"));
    }
    float l = 0.f;
    HELK_TRY(cuda_check(c, cudaMemcpyAsync(&l, c->mlp_loss, 4, cudaMemcpyDeviceToHost, c->stream), "surrogate"));
    HELK_TRY(helk_sync(c));
    last = (double)l / (double)(steps_per_epoch * batch);
  }
  if (final_loss) *final_loss = last;
  return HELK_OK;
}

helk_status helk_surrogate_eval(helk_ctx *c, int64_t n, const double *x, const double *y, double *k) {
  if (!c || n < 0 || (n > 0 && (!x || !y || !k))) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->mlp_p) return set_err(c, HELK_ERR_STATE, "surrogate: no network (call helk_surrogate_init)");
  HELK_TRY(bind_device(c));
  return cuda_check(c, launch_mlp_eval(c, c->mlp_p, n, x, y, k), "surrogate eval");
}

helk_status helk_surrogate_validate(helk_ctx *c, int32_t nx, int32_t ny, int32_t per_cell, double tol,
                                    uint8_t *mask_host, double *err_host) {
  if (!c || nx < 1 || ny < 1 || nx * ny > 65536 || per_cell < 1 || per_cell > 64 || !(tol > 0.0))
    return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->mlp_p) return set_err(c, HELK_ERR_STATE, "surrogate: no network (call helk_surrogate_init)");
  HELK_TRY(bind_device(c));
  const int ncell = nx * ny;
  double *err = nullptr;
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&err, (size_t)ncell * 12 + 16), "surrogate validate"));
  helk_status st = cuda_check(c, cudaMemsetAsync(err, 0, (size_t)ncell * 12 + 16, c->stream), "surrogate validate");
  if (st == HELK_OK) st = cuda_check(c, launch_mlp_validate(c, nx, ny, per_cell, err), "surrogate validate");
  std::vector<double> e(ncell);
  std::vector<unsigned int> cnt(ncell);
  if (st == HELK_OK) st = helk_sync(c);
  if (st == HELK_OK) st = cuda_check(c, cudaMemcpy(e.data(), err, ncell * 8, cudaMemcpyDeviceToHost), "validate");
  if (st == HELK_OK)
    st = cuda_check(c, cudaMemcpy(cnt.data(), err + ncell, ncell * 4, cudaMemcpyDeviceToHost), "validate");
  cudaFree(err);
  HELK_TRY(st);
  std::vector<uint32_t> bits((ncell + 31) / 32, 0u);
  for (int i = 0; i < ncell; ++i) {
    const bool ok = cnt[i] > 0 && e[i] <= tol;
    if (ok) bits[i >> 5] |= 1u << (i & 31);
    if (mask_host) mask_host[i] = ok ? 1 : 0;
    if (err_host) err_host[i] = cnt[i] > 0 ? e[i] : -1.0;
  }
  if (c->mlp_mask) cudaFree(c->mlp_mask);
  c->mlp_mask = nullptr;
  HELK_TRY(cuda_check(c, cudaMalloc((void **)&c->mlp_mask, bits.size() * 4), "surrogate mask"));
  HELK_TRY(cuda_check(c, cudaMemcpy(c->mlp_mask, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice), "mask"));
  c->mlp_mask_nx = nx;
  c->mlp_mask_ny = ny;
  if (c->squeue) {  // point the routing queue at the new mask
    SurrQueue q;
    HELK_TRY(cuda_check(c, cudaMemcpy(&q, c->squeue, sizeof q, cudaMemcpyDeviceToHost), "mask"));
    q.mask = c->mlp_mask;
    q.nx = nx;
    q.ny = ny;
    HELK_TRY(cuda_check(c, cudaMemcpy(c->squeue, &q, sizeof q, cudaMemcpyHostToDevice), "mask"));
  }
  return HELK_OK;
}

int64_t helk_launch_count(const helk_ctx *c) { return c ? c->launches : -1; }

int32_t helk_tile_candidates(int32_t precision, int32_t *out, int32_t max) {
  if (!out || (precision != HELK_PREC_F64 && precision != HELK_PREC_F32_KAHAN)) return 0;
  int cand[32];
  const int n = voigt_shape_candidates(precision, cand, 32);
  for (int i = 0; i < n && i < max; ++i) out[i] = cand[i];
  return n;
}

helk_status helk_tile_shape(int32_t precision, int32_t code, int32_t *points, int32_t *warps,
                            int32_t *lines_per_stage) {
  if (precision != HELK_PREC_F64 && precision != HELK_PREC_F32_KAHAN) return HELK_ERR_INVALID_ARG;
  int p = 0, w = 0, l = 0;
  if (!voigt_shape_info(precision, code, &p, &w, &l)) return HELK_ERR_INVALID_ARG;
  if (points) *points = p;
  if (warps) *warps = w;
  if (lines_per_stage) *lines_per_stage = l;
  return HELK_OK;
}

helk_status helk_set_tile(helk_ctx *c, int32_t precision, int64_t n, int32_t tile) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (precision != HELK_PREC_F64 && precision != HELK_PREC_F32_KAHAN)
    return set_err(c, HELK_ERR_INVALID_ARG, "set_tile: unknown precision");
  if (n < 1) return set_err(c, HELK_ERR_INVALID_ARG, "set_tile: n must be >= 1");
  const int prec = precision == HELK_PREC_F32_KAHAN ? 1 : 0;
  if (tile == 0) {
    c->tuned_tile[prec] = 0;
    return HELK_OK;
  }
  int cand[32];
  const int nc = voigt_shape_candidates(precision, cand, 32);
  bool ok = false;
  for (int i = 0; i < nc; ++i) ok = ok || cand[i] == tile;
  if (!ok) return set_err(c, HELK_ERR_INVALID_ARG, "set_tile: not a built tile shape");
  c->tuned_tile[prec] = tile;
  c->tuned_n[prec] = n;
  return HELK_OK;
}

helk_status helk_selftest_timeout(helk_ctx *c, int32_t limit_us) {
  if (!c || limit_us < 1 || limit_us > 10 * 1000 * 1000) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  HELK_TRY(bind_device(c));
  return cuda_check(c, launch_selftest_timeout(c, limit_us), "selftest");
}

helk_status helk_peak_probe(helk_ctx *c, int32_t kind, double *ops_per_s, double *ms_per_launch) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->err.clear();
  if (kind < HELK_PROBE_FFMA || kind > HELK_PROBE_MUFU_EX2 || !ops_per_s)
    return set_err(c, HELK_ERR_INVALID_ARG, "peak_probe: unknown kind or null output");
  HELK_TRY(bind_device(c));
  const int blocks = probe_blocks(c);
  HELK_TRY(ensure_buf(c, &c->tmp, &c->tmp_cap, (int64_t)blocks * 8, "peak probe"));
  cudaEvent_t e0, e1;
  HELK_TRY(cuda_check(c, cudaEventCreate(&e0), "peak probe"));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_check(c, cudaErrorUnknown, "peak probe");
  }
  // calibrate the loop length to ~20 ms a launch, then time three launches
  auto timed = [&](int iters, int reps, float *ms) -> helk_status {
    helk_status st = cuda_check(c, cudaEventRecord(e0, c->stream), "peak probe");
    for (int r = 0; r < reps && st == HELK_OK; ++r)
      st = cuda_check(c, launch_probe(c, kind, iters, blocks, c->tmp), "peak probe");
    if (st == HELK_OK) st = cuda_check(c, cudaEventRecord(e1, c->stream), "peak probe");
    if (st == HELK_OK) st = cuda_check(c, cudaEventSynchronize(e1), "peak probe");
    if (st == HELK_OK) st = cuda_check(c, cudaEventElapsedTime(ms, e0, e1), "peak probe");
    return st;
  };
  float ms = 0.f;
  int iters = 64;
  helk_status st = timed(iters, 1, &ms);  // warm-up
  for (int k = 0; k < 8 && st == HELK_OK && ms < 5.0f && iters < (1 << 22); ++k) {
    iters *= 4;
    st = timed(iters, 1, &ms);
  }
  if (st == HELK_OK && ms > 0.0f)
    iters = (int)std::min<double>((double)(1 << 24), std::max(64.0, iters * 20.0 / ms));
  const int reps = 3;
  if (st == HELK_OK) st = timed(iters, reps, &ms);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HELK_TRY(st);
  HELK_TRY(helk_sync(c));
  const double per_launch = ms / reps;
  const double ops = (double)blocks * probe_threads() * probe_ops_per_iter() * (double)iters *
                     ((kind == HELK_PROBE_FFMA || kind == HELK_PROBE_DFMA) ? 2.0 : 1.0);
  *ops_per_s = ops / (per_launch * 1e-3);
  if (ms_per_launch) *ms_per_launch = per_launch;
  return HELK_OK;
}

helk_status helk_set_profiling(helk_ctx *c, int32_t on) {
  if (!c) return HELK_ERR_INVALID_ARG;
  c->profiling = on != 0;
  for (int st = 0; st < HELK_NSTAGES; ++st) {
    c->ev_used[st] = 0;
    c->ev_overflow[st] = false;
  }
  return HELK_OK;
}

helk_status helk_stage_times(helk_ctx *c, double *ms, int64_t *count) {
  if (!c || !ms) return HELK_ERR_INVALID_ARG;
  HELK_TRY(bind_device(c));
  HELK_TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "stage_times"));
  for (int st = 0; st < HELK_NSTAGES; ++st) {
    double tot = 0.0;
    for (int64_t i = 0; i < c->ev_used[st]; ++i) {
      float t = 0.f;
      HELK_TRY(cuda_check(c, cudaEventElapsedTime(&t, c->ev[st][2 * i], c->ev[st][2 * i + 1]),
                          "stage_times"));
      tot += t;
    }
    ms[st] = tot;
    if (count) count[st] = c->ev_overflow[st] ? -c->ev_used[st] : c->ev_used[st];
  }
  return HELK_OK;
}

}  // extern "C"
