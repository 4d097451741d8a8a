// k_voigt.cu -- line-tiled Voigt opacity kernels (Sec. 2.3-2.5).
//
// Decomposition: one CTA owns one grid tile of BLOCK * nslot points
// (nslot <= PPT, chosen per call so that the tiles fill whole waves of
// resident CTAs); thread t owns points t, t+BLOCK, ... so each warp covers
// 32 consecutive points per slot (coalesced flush, and the method regions --
// which depend on |u| -- change at most at a few places per warp and line).
// The tile's candidate lines (a contiguous range of the nu0-ordered list) are
// staged through shared memory in chunks by 1-D bulk TMA copies, double
// buffered on two mbarriers.  Every point accumulates its lines in list order
// in registers; tiles own disjoint points, so there are no atomics and the
// result is deterministic.
//
// Two arithmetic forms:
//   k_voigt_f64  FP64 throughout; u and r^2 use explicitly rounded operations
//                so that the method chosen per point matches the FP64
//                definition bit for bit.
//   k_voigt_f32  FP32 profile evaluation on records with strengths scaled by
//                2^-E, Kahan-compensated FP32 accumulation per point, result
//                converted to FP64 and rescaled at the flush.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "helk_internal.cuh"

namespace helk {

constexpr long long WAIT_LIMIT = 1ll << 24;  // polls of a bulk-copy barrier

// ------------------------------------------------------------------------
// Algorithm 916 (Sec. 2.5), FP64.  K(x, y) for 0 <= x, x^2 + y^2 < 100:
//   K = e^{-x^2} erfcx(y) cos(2xy) + (2hx/pi) e^{-x^2} sin(xy) sinc(xy)
//     + (2h/pi) [ -y cos(2xy) e^{-x^2} S1 + (y/2)(S2 + S3) ],
//   S1 = sum e^{-(nh)^2}/((nh)^2+y^2)  (per line: sig1),
//   S2 + S3 = sum (e^{-(nh+x)^2} + e^{-(nh-x)^2}) / ((nh)^2 + y^2),
// the exponentials of S2/S3 advanced by the exact ratio recurrences
//   e^{-((n+1)h -+ x)^2} = e^{-(nh -+ x)^2} * R,  R <- R e^{-2h^2}.
// Only the terms within A916_TAIL of the Gaussian peaks are summed.
__device__ __forceinline__ void a916_range(double x, int &n0, int &n1) {
  n0 = (int)floor((x - A916_TAIL) / A916_H);
  if (n0 < 1) n0 = 1;
  n1 = (int)ceil((x + A916_TAIL) / A916_H);
}

__device__ __noinline__ double k916_f64(double x, double y, double erfcx_y, double sig1) {
  const double h = A916_H;
  const double ex2 = exp(-(x * x));
  const double xy = x * y;
  double s, c;
  sincos(xy, &s, &c);
  const double sinc = (xy == 0.0) ? 1.0 : s / xy;
  const double c2xy = c * c - s * s;
  int n0, n1;
  a916_range(x, n0, n1);
  const double q = 0.60653065971263342360;  // e^{-2h^2}
  const double nh = n0 * h;
  const double dm = nh - x, dp = nh + x;
  double E3 = exp(-(dm * dm));
  double R3 = exp(-(2.0 * h * dm + h * h));
  double E2 = exp(-(dp * dp));
  double R2 = exp(-(2.0 * h * dp + h * h));
  double s23 = 0.0;
  const double y2 = y * y;
  for (int n = n0; n <= n1; ++n) {
    const double nhn = n * h;
    s23 += (E2 + E3) / (nhn * nhn + y2);
    E3 *= R3;
    R3 *= q;
    E2 *= R2;
    R2 *= q;
  }
  double K = ex2 * erfcx_y * c2xy;
  K += (2.0 * h / PI) * x * ex2 * s * sinc;
  K += (2.0 * h / PI) * (0.5 * y * s23 - y * c2xy * ex2 * sig1);
  return K;
}

// The same series in FP32 (accurate expf/sincosf; recurrences start at the
// low end of the summed range, where the terms are ~e^{-38}, so nothing
// overflows or underflows in FP32).
__device__ __noinline__ float k916_f32(float x, float y, float erfcx_y, float sig1) {
  const float h = 0.5f;
  const float ex2 = expf(-(x * x));
  const float xy = x * y;
  float s, c;
  sincosf(xy, &s, &c);
  const float sinc = (xy == 0.0f) ? 1.0f : s / xy;
  const float c2xy = c * c - s * s;
  int n0 = (int)floorf((x - 6.2f) * 2.0f);
  if (n0 < 1) n0 = 1;
  const int n1 = (int)ceilf((x + 6.2f) * 2.0f);
  const float q = 0.60653065971f;  // e^{-2h^2}
  const float nh = n0 * h;
  const float dm = nh - x, dp = nh + x;
  float E3 = expf(-(dm * dm));
  float R3 = expf(-(2.0f * h * dm + h * h));
  float E2 = expf(-(dp * dp));
  float R2 = expf(-(2.0f * h * dp + h * h));
  float s23 = 0.0f;
  const float y2 = y * y;
  for (int n = n0; n <= n1; ++n) {
    const float nhn = n * h;
    s23 += __fdividef(E2 + E3, fmaf(nhn, nhn, y2));
    E3 *= R3;
    R3 *= q;
    E2 *= R2;
    R2 *= q;
  }
  const float k2h = 0.31830988618f;  // 2h/pi
  float K = ex2 * erfcx_y * c2xy;
  K += k2h * x * ex2 * s * sinc;
  K += k2h * (0.5f * y * s23 - y * c2xy * ex2 * sig1);
  return K;
}

// ------------------------------------------------------ line staging ----
// Double-buffered bulk-copy pipeline over the line range [l0, l1).
template <typename Rec, int LCH>
struct LineStager {
  Rec (*sl)[LCH];
  uint32_t mb[2];
  int l0, l1, nch;
  const Rec *rec;

  __device__ void init(Rec (*buf)[LCH], unsigned long long *mbar, const Rec *r, int a, int b) {
    sl = buf;
    rec = r;
    l0 = a;
    l1 = b;
    nch = (l1 - l0 + LCH - 1) / LCH;
    mb[0] = smem_addr(&mbar[0]);
    mb[1] = smem_addr(&mbar[1]);
    if (threadIdx.x == 0) {
      mbar_init(mb[0], 1);
      mbar_init(mb[1], 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && nch > 0) issue(0);
  }
  __device__ int count(int ch) const { return min(LCH, l1 - l0 - ch * LCH); }
  __device__ void issue(int ch) {
    tma_load_1d(smem_addr(&sl[ch & 1][0]), rec + l0 + ch * LCH, (uint32_t)(count(ch) * sizeof(Rec)),
                mb[ch & 1]);
  }
  // Prefetch chunk ch+1, wait for chunk ch.  Returns false (for every thread)
  // if the wait gave up; the caller must then return.
  __device__ bool acquire(int ch, int *flags) {
    if (threadIdx.x == 0 && ch + 1 < nch) issue(ch + 1);
    const bool ok = mbar_wait_bounded(mb[ch & 1], (ch >> 1) & 1, flags, WAIT_LIMIT);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0 && ch + 1 < nch)
        mbar_wait_bounded(mb[(ch + 1) & 1], ((ch + 1) >> 1) & 1, flags, WAIT_LIMIT);
      return false;
    }
    return true;
  }
};

// ------------------------------------------------------------ FP64 form --
template <int BLOCK, int PPT, int LCH, bool COUNT>
__global__ void __launch_bounds__(BLOCK)
    k_voigt_f64(const LineRec64 *__restrict__ rec, const int32_t *__restrict__ tlo,
                const int32_t *__restrict__ thi, double nu_min, double dnu, int ngrid, int nslot,
                double weight, int accumulate, double *__restrict__ kappa, DevStats *st) {
  __shared__ __align__(128) LineRec64 sl[2][LCH];
  __shared__ __align__(8) unsigned long long mbar[2];
  const int tid = threadIdx.x;
  const int tile_len = BLOCK * nslot;
  const int base = blockIdx.x * tile_len;
  double nu[PPT], acc[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = base + tid + k * BLOCK;
    nu[k] = __dadd_rn(nu_min, __dmul_rn((double)i, dnu));
    acc[k] = 0.0;
  }
  unsigned long long cnt[4] = {0, 0, 0, 0};
  LineStager<LineRec64, LCH> stg;
  stg.init(sl, mbar, rec, tlo[blockIdx.x], thi[blockIdx.x]);
  for (int ch = 0; ch < stg.nch; ++ch) {
    if (!stg.acquire(ch, &st->err_flags)) return;
    const int cnum = stg.count(ch);
    const LineRec64 *buf = sl[ch & 1];
    for (int j = 0; j < cnum; ++j) {
      const LineRec64 &L = buf[j];
      const int ilo = L.ilo, ihi = L.ihi;
      if (ihi < base || ilo >= base + tile_len || ihi < ilo) continue;
      const bool full = (ilo <= base) && (ihi >= base + tile_len - 1);
      const double nu0p = L.nu0p, ku = L.ku, a = L.a, a2 = L.a2, Sp = L.Sp;
      const double P1 = Sp * a * INV_SQRTPI;           // GH1: (a/pi) sqrt(pi)
      const double P3 = Sp * a * (SQRTPI / 6.0) / PI;  // GH3 outer weight
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (k >= nslot) break;
        const int i = base + tid + k * BLOCK;
        if (full || (i >= ilo && i <= ihi)) {
          const double u = __dmul_rn(__dsub_rn(nu[k], nu0p), ku);
          const double r2 = __dadd_rn(__dmul_rn(u, u), a2);
          double v;
          if (r2 >= R2_GH1) {
            v = P1 / r2;
            if (COUNT) cnt[2]++;
          } else if (r2 >= R2_GH3) {
            // (a/pi)[w0/d0 + w1/d1 + w1/d2], w0 = 4 w1, one division
            const double um = u - GH3_T, up = u + GH3_T;
            const double d1 = um * um + a2, d2 = up * up + a2;
            const double p = d1 * d2;
            const double num = 4.0 * p + r2 * (d1 + d2);
            v = P3 * (num / (r2 * p));
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
      if ((tid & 31) == 0 && v) atomicAdd(&st->region[r], v);
    }
  }
}

// ------------------------------------------------------------ FP32 form --
template <int BLOCK, int PPT, int LCH, bool COUNT>
__global__ void __launch_bounds__(BLOCK)
    k_voigt_f32(const LineRec32 *__restrict__ rec, const int32_t *__restrict__ tlo,
                const int32_t *__restrict__ thi, int ngrid, int nslot, double weight,
                int accumulate, double *__restrict__ kappa, DevStats *st) {
  __shared__ __align__(128) LineRec32 sl[2][LCH];
  __shared__ __align__(8) unsigned long long mbar[2];
  const int tid = threadIdx.x;
  const int tile_len = BLOCK * nslot;
  const int base = blockIdx.x * tile_len;
  float sum[PPT], comp[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    sum[k] = 0.0f;
    comp[k] = 0.0f;
  }
  unsigned long long cnt[4] = {0, 0, 0, 0};
  LineStager<LineRec32, LCH> stg;
  stg.init(sl, mbar, rec, tlo[blockIdx.x], thi[blockIdx.x]);
  for (int ch = 0; ch < stg.nch; ++ch) {
    if (!stg.acquire(ch, &st->err_flags)) return;
    const int cnum = stg.count(ch);
    const LineRec32 *buf = sl[ch & 1];
    for (int j = 0; j < cnum; ++j) {
      const LineRec32 &L = buf[j];
      const int ilo = L.ilo, ihi = L.ihi;
      if (ihi < base || ilo >= base + tile_len || ihi < ilo) continue;
      const bool full = (ilo <= base) && (ihi >= base + tile_len - 1);
      const float beta = L.beta, nphi = -L.phi_k, a2 = L.a2, P1 = L.P1, P3 = L.P3;
      // (i - c) for this thread's first point; exact in FP32 (|i - c| < 2^24
      // whenever the point is inside the window)
      const float d0 = (float)(base + tid - L.c);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (k >= nslot) break;
        const int i = base + tid + k * BLOCK;
        if (full || (i >= ilo && i <= ihi)) {
          const float u = fmaf(d0 + (float)(k * BLOCK), beta, nphi);
          const float r2 = fmaf(u, u, a2);
          float v;
          if (r2 >= 1.0e6f) {
            v = __fdividef(P1, r2);
            if (COUNT) cnt[2]++;
          } else if (r2 >= 100.0f) {
            const float um = u - 1.2247448714f, up = u + 1.2247448714f;
            const float d1 = fmaf(um, um, a2), d2 = fmaf(up, up, a2);
            const float p = d1 * d2;
            const float num = fmaf(4.0f, p, r2 * (d1 + d2));
            v = P3 * __fdividef(num, r2 * p);
            if (COUNT) cnt[1]++;
          } else {
            v = L.Sp * k916_f32(fabsf(u), L.a, L.erfcx_a, L.sig1);
            if (COUNT) {
              int n0, n1;
              a916_range(fabs((double)u), n0, n1);
              cnt[0]++;
              cnt[3] += (unsigned long long)(n1 - n0 + 1);
            }
          }
          // Kahan-compensated accumulation
          const float yk = v - comp[k];
          const float t = sum[k] + yk;
          comp[k] = (t - sum[k]) - yk;
          sum[k] = t;
        }
      }
    }
    __syncthreads();
  }
  const double scale = ldexp(weight, st->scale_exp);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = base + tid + k * BLOCK;
    if (k < nslot && i < ngrid) {
      const double v = scale * ((double)sum[k] - (double)comp[k]);
      kappa[i] = accumulate ? kappa[i] + v : v;
    }
  }
  if (COUNT) {
    for (int r = 0; r < 4; ++r) {
      unsigned long long v = cnt[r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0 && v) atomicAdd(&st->region[r], v);
    }
  }
}

// --------------------------------------------------------------- launch --
constexpr int F64_BLOCK = 256, F64_PPT = 8, F64_LCH = 64;
constexpr int F32_BLOCK = 256, F32_PPT = 16, F32_LCH = 128;

template <typename K>
static int resident_ctas(helk_ctx *c, K kern, int block) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return occ * c->num_sms;
}

// Pick nslot <= PPT so that ceil(n / (BLOCK nslot)) tiles fill whole waves
// of `slots` resident CTAs as evenly as possible, preferring long tiles
// (each (line, tile) pair has a fixed setup cost of about one slot).
static int pick_nslot(int64_t n, int block, int ppt, int slots) {
  int best = ppt;
  double best_score = -1.0;
  for (int p = ppt; p >= 1; --p) {
    const int64_t ntiles = (n + (int64_t)block * p - 1) / ((int64_t)block * p);
    const double waves = (double)ntiles / slots;
    const double eff = waves / ceil(waves);
    const double score = eff * p / (p + 1.0);
    if (score > best_score + 1e-9) {
      best_score = score;
      best = p;
    }
  }
  return best;
}

int voigt_tile_len(helk_ctx *c, int precision, int count, int64_t n) {
  if (precision == HELK_PREC_F32_KAHAN) {
    const int slots = count ? resident_ctas(c, k_voigt_f32<F32_BLOCK, F32_PPT, F32_LCH, true>, F32_BLOCK)
                            : resident_ctas(c, k_voigt_f32<F32_BLOCK, F32_PPT, F32_LCH, false>, F32_BLOCK);
    return F32_BLOCK * pick_nslot(n, F32_BLOCK, F32_PPT, slots);
  }
  const int slots = count ? resident_ctas(c, k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, true>, F64_BLOCK)
                          : resident_ctas(c, k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, false>, F64_BLOCK);
  return F64_BLOCK * pick_nslot(n, F64_BLOCK, F64_PPT, slots);
}

cudaError_t launch_voigt(helk_ctx *c, const helk_grid &g, const helk_opts &o, double *kappa,
                         int tile_len, int64_t ntiles) {
  const unsigned grid = (unsigned)ntiles;
  if (o.precision == HELK_PREC_F32_KAHAN) {
    const int nslot = tile_len / F32_BLOCK;
    if (o.count_regions)
      k_voigt_f32<F32_BLOCK, F32_PPT, F32_LCH, true><<<grid, F32_BLOCK, 0, c->stream>>>(
          c->rec32, c->tile_lo, c->tile_hi, (int)g.n, nslot, o.weight, o.accumulate, kappa, c->stats);
    else
      k_voigt_f32<F32_BLOCK, F32_PPT, F32_LCH, false><<<grid, F32_BLOCK, 0, c->stream>>>(
          c->rec32, c->tile_lo, c->tile_hi, (int)g.n, nslot, o.weight, o.accumulate, kappa, c->stats);
  } else {
    const int nslot = tile_len / F64_BLOCK;
    if (o.count_regions)
      k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, true><<<grid, F64_BLOCK, 0, c->stream>>>(
          c->rec64, c->tile_lo, c->tile_hi, g.nu_min, g.dnu, (int)g.n, nslot, o.weight, o.accumulate,
          kappa, c->stats);
    else
      k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, false><<<grid, F64_BLOCK, 0, c->stream>>>(
          c->rec64, c->tile_lo, c->tile_hi, g.nu_min, g.dnu, (int)g.n, nslot, o.weight, o.accumulate,
          kappa, c->stats);
  }
  return cudaGetLastError();
}

}  // namespace helk
