// k_voigt64.cu -- the FP64 form of the line-tiled Voigt opacity kernel
// (Sec. 2.3-2.4): FP64 throughout; u and r^2 use explicitly rounded
// operations so that the method chosen per point matches the FP64 definition
// bit for bit.
//
// Decomposition: one CTA owns one grid tile of BLOCK * nslot points
// (nslot <= PPT, chosen per call so that the tiles fill whole waves of
// resident CTAs); thread t owns points t, t+BLOCK, ... so each warp covers
// 32 consecutive points per slot.  The tile's candidate lines (a contiguous
// range of the nu0-ordered list) are staged through shared memory in chunks
// by 1-D bulk TMA copies, double buffered on two mbarriers.  Every point
// accumulates its lines in list order in registers; tiles own disjoint
// points, so there are no atomics and the result is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "helk_internal.cuh"
#include "voigt_common.cuh"
#include "voigt_core.cuh"

namespace helk {

// Reciprocal of a double x >= 100: FP32 hardware seed (relative error
// < 2^-22) refined by one Newton step, relative error < 1e-13 -- far inside
// the 1e-9 budget of the FP64 form, at a fraction of the cost of an IEEE
// division on the FP64 pipe.  Beyond the FP32 range the seed is 0 and the
// division is done exactly.
__device__ __forceinline__ double rcp64(double x) {
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)x));
  if (rf == 0.0f) return 1.0 / x;
  const double r = (double)rf;
  return fma(r, fma(-x, r, 1.0), r);
}

// ------------------------------------------------------ line staging ----
// Double-buffered bulk-copy pipeline over a line range [l0, l1).  The two
// mbarriers are initialised once per CTA; chunks are numbered across all the
// ranges a persistent CTA processes (gch), which fixes each chunk's buffer
// (gch & 1) and barrier phase ((gch >> 1) & 1).
template <typename Rec, int LCH>
struct LineStager {
  Rec (*sl)[LCH];
  uint32_t mb[2];
  int l0, l1, nch;
  uint32_t gbase;  // global number of this range's chunk 0
  const Rec *rec;

  __device__ void init(Rec (*buf)[LCH], unsigned long long *mbar) {
    sl = buf;
    gbase = 0;
    nch = 0;
    mb[0] = smem_addr(&mbar[0]);
    mb[1] = smem_addr(&mbar[1]);
    if (threadIdx.x == 0) {
      mbar_init(mb[0], 1);
      mbar_init(mb[1], 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  // Start a new range; every thread must have finished the previous one.
  __device__ void begin(const Rec *r, int a, int b) {
    gbase += nch;
    rec = r;
    l0 = a;
    l1 = b;
    nch = (l1 - l0 + LCH - 1) / LCH;
    if (threadIdx.x == 0 && nch > 0) issue(0);
  }
  __device__ int count(int ch) const { return min(LCH, l1 - l0 - ch * LCH); }
  __device__ const Rec *buffer(int ch) const { return sl[(gbase + ch) & 1]; }
  __device__ void issue(int ch) {
    const uint32_t g = gbase + ch;
    tma_load_1d(smem_addr(&sl[g & 1][0]), rec + l0 + ch * LCH, (uint32_t)(count(ch) * sizeof(Rec)),
                mb[g & 1]);
  }
  // Prefetch chunk ch+1, wait for chunk ch.  Returns false (for every thread)
  // if the wait gave up; the caller must then return.
  __device__ bool acquire(int ch, int *flags) {
    if (threadIdx.x == 0 && ch + 1 < nch) issue(ch + 1);
    const uint32_t g = gbase + ch;
    const bool ok = mbar_wait_bounded(mb[g & 1], (g >> 1) & 1, flags, WAIT_LIMIT_NS);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0 && ch + 1 < nch)
        mbar_wait_bounded(mb[(g + 1) & 1], ((g + 1) >> 1) & 1, flags, WAIT_LIMIT_NS);
      return false;
    }
    return true;
  }
};

// Next (condition, tile) item of a persistent CTA: -1 when none is left.
__device__ __forceinline__ int next_item(DevStats *st, int nitems, int *s_item) {
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(&st->tile_counter, 1u);
  __syncthreads();
  const int item = *s_item;
  __syncthreads();
  return item < nitems ? item : -1;
}

// ------------------------------------------------------------ FP64 form --
// Persistent: each CTA takes (condition, tile) items until none are left;
// items of the condition with the most evaluations come first.
template <int BLOCK, int PPT, int LCH, bool COUNT>
__global__ void __launch_bounds__(BLOCK)
    k_voigt_f64(const LineRec64 *__restrict__ rec_all, int64_t nlines,
                const int32_t *__restrict__ tlo_all, const int32_t *__restrict__ thi_all,
                int64_t ntiles, const int *__restrict__ cond_order, int n_cond, double nu_min,
                double dnu, int ngrid, int nslot, double weight, int accumulate,
                double *__restrict__ kappa_all, CondStats *cst, DevStats *st) {
  __shared__ __align__(128) LineRec64 sl[2][LCH];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const int tile_len = BLOCK * nslot;
  LineStager<LineRec64, LCH> stg;
  stg.init(sl, mbar);
  const int nitems = (int)(ntiles * n_cond);
  for (int item = next_item(st, nitems, &s_item); item >= 0; item = next_item(st, nitems, &s_item)) {
  const int cond = cond_order[item / ntiles];
  const int64_t tile = item % ntiles;
  const LineRec64 *rec = rec_all + cond * nlines;
  double *kappa = kappa_all + (int64_t)cond * ngrid;
  const int base = (int)(tile * tile_len);
  double nu[PPT], acc[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = base + tid + k * BLOCK;
    nu[k] = __dadd_rn(nu_min, __dmul_rn((double)i, dnu));
    acc[k] = 0.0;
  }
  unsigned long long cnt[4] = {0, 0, 0, 0};
  stg.begin(rec, tlo_all[cond * ntiles + tile], thi_all[cond * ntiles + tile]);
  for (int ch = 0; ch < stg.nch; ++ch) {
    if (!stg.acquire(ch, &st->err_flags)) return;
    const int cnum = stg.count(ch);
    const LineRec64 *buf = stg.buffer(ch);
    for (int j = 0; j < cnum; ++j) {
      const LineRec64 &L = buf[j];
      const int ilo = L.ilo, ihi = L.ihi;
      if (ihi < base || ilo >= base + tile_len || ihi < ilo) continue;
      const bool full = (ilo <= base) && (ihi >= base + tile_len - 1);
      const double nu0p = L.nu0p, ku = L.ku, a = L.a, a2 = L.a2, Sp = L.Sp;
      const double P1 = Sp * a * INV_SQRTPI;           // GH1: (a/pi) sqrt(pi)
      // GH3 as a rational function of r2 alone (u^2 = r2 - a^2):
      //   (a w1/pi)[4/r2 + 2q/p] = (c3 r2^2 + c45 r2 + c2) / (r2 (r2 (r2 - 3) + C)),
      // q = r2 + 3/2, p = r2 (r2 - 3) + C, C = 9/4 + 6 a^2, with the line's
      // factor P3h = 2 a w1 S'/pi in c3 = 3 P3h, c45 = -9/2 P3h, c2 = 2C P3h
      const double P3h = 2.0 * (Sp * a * (SQRTPI / 6.0) / PI);
      const double C3 = fma(6.0, a2, 2.25);
      const double c3 = 3.0 * P3h, c45 = -4.5 * P3h, c2 = 2.0 * C3 * P3h;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (k >= nslot) break;
        const int i = base + tid + k * BLOCK;
        if (full || (i >= ilo && i <= ihi)) {
          const double u = __dmul_rn(__dsub_rn(nu[k], nu0p), ku);
          const double r2 = __dadd_rn(__dmul_rn(u, u), a2);
          double v;
          if (r2 >= R2_GH1) {
            v = P1 * rcp64(r2);
            if (COUNT) cnt[2]++;
          } else if (r2 >= R2_GH3) {
            const double p = fma(r2, r2 - 3.0, C3);
            v = fma(r2, fma(c3, r2, c45), c2) * rcp64(r2 * p);
            if (COUNT) cnt[1]++;
          } else {
            v = Sp * k916_f64(fabs(u), a, L.erfcx_a, L.sig1);
            if (COUNT) {
              int n0, n1;
              a916_range(fabs(u), n0, n1);
              cnt[0]++;
              cnt[3] += (unsigned long long)(n1 - n0 + 1);
            }
          }
          acc[k] += v;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = base + tid + k * BLOCK;
    if (k < nslot && i < ngrid) {
      const double v = weight * acc[k];
      kappa[i] = accumulate ? kappa[i] + v : v;
    }
  }
  if (COUNT) {
    for (int r = 0; r < 4; ++r) {
      unsigned long long v = cnt[r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0 && v) atomicAdd(&cst[cond].region[r], v);
    }
  }
  }
}

// ------------------------------------------------- failure-detection test --
// One thread waits, with the same bounded wait as the Voigt kernels, on an
// mbarrier phase that nothing completes; after `limit_ns` nanoseconds of the
// global timer it sets the timeout flag and returns.
__global__ void k_selftest_timeout(DevStats *st, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long mbar;
  if (threadIdx.x != 0) return;
  const uint32_t mb = smem_addr(&mbar);
  mbar_init(mb, 1);
  fence_mbar_init();
  mbar_wait_bounded(mb, 0, &st->err_flags, limit_ns);
}

cudaError_t launch_selftest_timeout(helk_ctx *c, int limit_us) {
  ++c->launches;
  k_selftest_timeout<<<1, 32, 0, c->stream>>>(c->stats, (unsigned long long)limit_us * 1000ull);
  return cudaGetLastError();
}

// --------------------------------------------------------------- launch --
constexpr int F64_BLOCK = 256, F64_PPT = 8, F64_LCH = 64;

// Pick nslot <= ppt so that ceil(n / (block nslot)) tiles fill whole waves
// of `slots` resident CTAs as evenly as possible, preferring long tiles
// (each (line, tile) pair has a fixed setup cost of about one slot).
static double tile_score(int64_t n, int block, int p, int slots) {
  const int64_t ntiles = (n + (int64_t)block * p - 1) / ((int64_t)block * p);
  const double waves = (double)ntiles / slots;
  return waves / ceil(waves) * p / (p + 1.0);
}

static int pick_nslot(int64_t n, int block, int ppt, int slots) {
  int best = ppt;
  double best_score = -1.0;
  for (int p = ppt; p >= 1; --p) {
    const double score = tile_score(n, block, p, slots);
    if (score > best_score + 1e-9) {
      best_score = score;
      best = p;
    }
  }
  return best;
}

// FP64 shapes: the code is the slots per warp (1..F64_PPT) of 8-warp CTAs
// with 64-line stages; the autotuner times 4, 6 and 8.
bool f64_shape_info(int code, int *points, int *warps, int *lines_per_stage) {
  if (code < 1 || code > F64_PPT) return false;
  if (points) *points = F64_BLOCK * code;
  if (warps) *warps = F64_BLOCK / 32;
  if (lines_per_stage) *lines_per_stage = F64_LCH;
  return true;
}

int f64_shape_candidates(int *out, int max) {
  int n = 0;
  const int f64_choices[] = {4, 6, 8};
  for (int p : f64_choices)
    if (n < max) out[n++] = p;
  return n;
}

int f64_shape(helk_ctx *c, int count, int64_t n) {
  const int slots = count ? resident_ctas(c, k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, true>, F64_BLOCK)
                          : resident_ctas(c, k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, false>, F64_BLOCK);
  return pick_nslot(n, F64_BLOCK, F64_PPT, slots);
}

cudaError_t launch_voigt_f64(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o, double *kappa,
                             int shape, int64_t ntiles) {
  const int64_t nitems = ntiles * n_cond;
  const int nslot = shape;
  if (nslot < 1 || nslot > F64_PPT) return cudaErrorInvalidValue;
  if (o.count_regions) {
    auto kern = k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, true>;
    ++c->launches;
    kern<<<persistent_grid(c, kern, F64_BLOCK, nitems), F64_BLOCK, 0, c->stream>>>(
        c->rec64, c->nlines, c->tile_lo, c->tile_hi, ntiles, c->cond_order, n_cond, g.nu_min, g.dnu,
        (int)g.n, nslot, o.weight, o.accumulate, kappa, c->cstats, c->stats);
  } else {
    auto kern = k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, false>;
    ++c->launches;
    kern<<<persistent_grid(c, kern, F64_BLOCK, nitems), F64_BLOCK, 0, c->stream>>>(
        c->rec64, c->nlines, c->tile_lo, c->tile_hi, ntiles, c->cond_order, n_cond, g.nu_min, g.dnu,
        (int)g.n, nslot, o.weight, o.accumulate, kappa, c->cstats, c->stats);
  }
  return cudaGetLastError();
}

}  // namespace helk
