// k_voigt.cu -- line-tiled Voigt opacity kernels (Sec. 2.3-2.5).
//
// Decomposition: one CTA owns one grid tile of BLOCK*PPT points; thread t
// owns points t, t+BLOCK, ... so each warp covers 32 consecutive points per
// slot (coalesced flush, and the method regions -- which depend on |u| --
// change at most at a few places per warp and line).  The tile's candidate
// lines (a contiguous range of the nu0-ordered list) are staged through
// shared memory in chunks by 1-D bulk TMA copies, double buffered on two
// mbarriers.  Every point accumulates its lines in list order in registers;
// tiles own disjoint points, so there are no atomics and the result is
// deterministic.
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
__device__ __noinline__ double k916_f64(double x, double y, double erfcx_y, double sig1) {
  const double h = A916_H;
  const double ex2 = exp(-(x * x));
  const double xy = x * y;
  double s, c;
  sincos(xy, &s, &c);
  const double sinc = (xy == 0.0) ? 1.0 : s / xy;
  const double c2xy = c * c - s * s;
  int n0 = (int)floor((x - A916_TAIL) / h);
  if (n0 < 1) n0 = 1;
  const int n1 = (int)ceil((x + A916_TAIL) / h);
  const double q = 0.60653065971263342360;  // e^{-2h^2}
  double nh = n0 * h;
  double dm = nh - x, dp = nh + x;
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

template <int BLOCK, int PPT, int LCH, bool COUNT>
__global__ void __launch_bounds__(BLOCK)
    k_voigt_f64(const LineRec64 *__restrict__ rec, const int32_t *__restrict__ tlo,
                const int32_t *__restrict__ thi, double nu_min, double dnu, int ngrid,
                double weight, int accumulate, double *__restrict__ kappa, DevStats *st) {
  constexpr int TILE = BLOCK * PPT;
  __shared__ __align__(128) LineRec64 sl[2][LCH];
  __shared__ __align__(8) unsigned long long mbar[2];
  const int tid = threadIdx.x;
  const int base = blockIdx.x * TILE;
  double nu[PPT], acc[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = base + tid + k * BLOCK;
    nu[k] = __dadd_rn(nu_min, __dmul_rn((double)i, dnu));
    acc[k] = 0.0;
  }
  unsigned long long cnt[4] = {0, 0, 0, 0};
  const int l0 = tlo[blockIdx.x], l1 = thi[blockIdx.x];
  const int nch = (l1 - l0 + LCH - 1) / LCH;
  const uint32_t mb0 = smem_addr(&mbar[0]), mb1 = smem_addr(&mbar[1]);
  if (tid == 0) {
    mbar_init(mb0, 1);
    mbar_init(mb1, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && nch > 0) {
    const int c0 = min(LCH, l1 - l0);
    tma_load_1d(smem_addr(&sl[0][0]), rec + l0, (uint32_t)c0 * sizeof(LineRec64), mb0);
  }
  for (int ch = 0; ch < nch; ++ch) {
    const int buf = ch & 1;
    if (tid == 0 && ch + 1 < nch) {
      const int cn = min(LCH, l1 - l0 - (ch + 1) * LCH);
      tma_load_1d(smem_addr(&sl[buf ^ 1][0]), rec + l0 + (ch + 1) * LCH,
                  (uint32_t)cn * sizeof(LineRec64), buf ? mb0 : mb1);
    }
    const bool ok = mbar_wait_bounded(buf ? mb1 : mb0, (ch >> 1) & 1, &st->err_flags, WAIT_LIMIT);
    if (__syncthreads_or(!ok)) {
      // give the copy still in flight (if any) a bounded chance to land
      if (tid == 0 && ch + 1 < nch)
        mbar_wait_bounded(buf ? mb0 : mb1, ((ch + 1) >> 1) & 1, &st->err_flags, WAIT_LIMIT);
      return;
    }
    const int cnum = min(LCH, l1 - l0 - ch * LCH);
    for (int j = 0; j < cnum; ++j) {
      const LineRec64 &L = sl[buf][j];
      const int ilo = L.ilo, ihi = L.ihi;
      if (ihi < base || ilo >= base + TILE || ihi < ilo) continue;
      const bool full = (ilo <= base) && (ihi >= base + TILE - 1);
      const double nu0p = L.nu0p, ku = L.ku, a = L.a, a2 = L.a2, Sp = L.Sp;
      const double P1 = Sp * a * INV_SQRTPI;           // GH1: (a/pi) sqrt(pi)
      const double P3 = Sp * a * (SQRTPI / 6.0) / PI;  // GH3 outer weight
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
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
              cnt[0]++;
              const double x = fabs(u);
              int n0 = (int)floor((x - A916_TAIL) / A916_H);
              if (n0 < 1) n0 = 1;
              cnt[3] += (unsigned long long)((int)ceil((x + A916_TAIL) / A916_H) - n0 + 1);
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
    if (i < ngrid) {
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

constexpr int F64_BLOCK = 256, F64_PPT = 8, F64_LCH = 64;

int voigt_tile_points(int precision) {
  (void)precision;
  return F64_BLOCK * F64_PPT;
}

cudaError_t launch_voigt(helk_ctx *c, const helk_grid &g, const helk_opts &o, double *kappa,
                         int64_t ntiles) {
  if (o.count_regions)
    k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, true><<<(unsigned)ntiles, F64_BLOCK, 0, c->stream>>>(
        c->rec64, c->tile_lo, c->tile_hi, g.nu_min, g.dnu, (int)g.n, o.weight, o.accumulate, kappa,
        c->stats);
  else
    k_voigt_f64<F64_BLOCK, F64_PPT, F64_LCH, false><<<(unsigned)ntiles, F64_BLOCK, 0, c->stream>>>(
        c->rec64, c->tile_lo, c->tile_hi, g.nu_min, g.dnu, (int)g.n, o.weight, o.accumulate, kappa,
        c->stats);
  return cudaGetLastError();
}

}  // namespace helk
