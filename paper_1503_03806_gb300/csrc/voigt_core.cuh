// voigt_core.cuh -- device functions of Algorithm 916 shared by the Voigt
// kernels and the surrogate's training-target kernel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "helk_internal.cuh"

namespace helk {

// ------------------------------------------------------------------------
// Algorithm 916 (Sec. 2.4), FP64.  K(x, y) for 0 <= x, x^2 + y^2 < 100:
//   K = e^{-x^2} erfcx(y) cos(2xy) + (2hx/pi) e^{-x^2} sin(xy) sinc(xy)
//     + (2h/pi) [ -y cos(2xy) e^{-x^2} S1 + (y/2)(S2 + S3) ],
//   S1 = sum e^{-(nh)^2}/((nh)^2+y^2)  (per line: sig1),
//   S2 + S3 = sum (e^{-(nh+x)^2} + e^{-(nh-x)^2}) / ((nh)^2 + y^2),
// the exponentials of S2/S3 advanced by the exact ratio recurrences
//   e^{-((n+1)h -+ x)^2} = e^{-(nh -+ x)^2} * R,  R <- R e^{-2h^2}.
// Only the terms within A916_TAIL of the Gaussian peaks are summed.
static __device__ __forceinline__ void a916_range(double x, int &n0, int &n1) {
  n0 = (int)floor((x - A916_TAIL) / A916_H);
  if (n0 < 1) n0 = 1;
  n1 = (int)ceil((x + A916_TAIL) / A916_H);
}

static __device__ __noinline__ double k916_f64(double x, double y, double erfcx_y, double sig1) {
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

// The same series in FP32.  Only the terms within
// A916_TAIL_F32 = 4.3 of the Gaussian peaks are summed (each dropped term is
// below e^{-18.49} = 9.3e-9 of its weight): the truncation is below 3e-9 of K
// over x^2 + y^2 < 100, y >= 1e-8 (against the exact w(z), in FP64), under
// FP32 resolution.  Every partial sum and factor of the FP32 series stays
// within the FP32 normal range (factors e^{-t^2/4} >= 4e-32, ratios <= 74,
// partial sums of Horner's rule <= ~1e9).
constexpr float A916_TAIL_F32 = 4.3f;
// n in [2(x - 4.3), 2(x + 4.3)], an interval of length 17.2: at most 18 terms
constexpr int A916_TERMS_F32 = 18;
// S2 terms e^{-(nh+x)^2} within the window have nh < 4.3: n <= 8
constexpr int A916_S2_TERMS_F32 = 8;

static __device__ __forceinline__ void a916_range_f32(float x, int &n0, int &n1) {
  n0 = (int)ceilf((x - A916_TAIL_F32) * 2.0f);
  if (n0 < 1) n0 = 1;
  n1 = (int)floorf((x + A916_TAIL_F32) * 2.0f);
}

// The series weights 1/((nh)^2 + y^2) of one line, n = 1..A916_NMAX_F32:
// every term of a window within A916_TAIL_F32 of x < 10 has
// n <= 2 (10 + 4.3) < A916_NMAX_F32.  Lane l of a warp computes n = l + 1,
// so a warp fills a line's table with one reciprocal a lane.
constexpr int A916_NMAX_F32 = 29;
static __device__ __forceinline__ float a916_weight_f32(int n, float y2) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaf((float)(n * n), 0.25f, y2)));
  return r;
}

// e^{-t^2/4}, t = 0 .. A916_TERMS_F32 - 1, rounded to FP32: with h = 1/2 the
// Gaussian factor of the t-th term past a window's first,
// e^{-(d + t h)^2} = e^{-d^2} (e^{-d})^t e^{-t^2/4}.
__device__ constexpr float A916_GAUSS_F32[A916_TERMS_F32] = {
    0x1.0p+0f,        0x1.8ebefap-1f,   0x1.78b564p-2f,   0x1.afb718p-4f,   0x1.2c155cp-6f,
    0x1.fa0e96p-10f,  0x1.02cf22p-13f,  0x1.411fb0p-18f,  0x1.e355bcp-24f,  0x1.b93de2p-30f,
    0x1.e8a37ap-37f,  0x1.4835bep-44f,  0x1.0b6c3ap-52f,  0x1.085194p-61f,  0x1.3ce9bap-71f,
    0x1.ccee16p-82f,  0x1.969d48p-93f,  0x1.b31fc8p-105f};

// Algorithm 916 in FP32 (accurate expf/sincosf) with the line's series
// weights from a table, w[n - 1] = 1/((nh)^2 + y^2).  Each series is a
// polynomial in the ratio of neighbouring peaks: with d the offset of the
// window's first term, sum_t e^{-(d + t h)^2} w_t = e^{-d^2} sum_t c_t rho^t,
// rho = e^{-d}, c_t = e^{-t^2/4} w_t, evaluated by Horner's rule from the
// last term (one multiply and one FMA a term; every partial sum positive).
static __device__ __forceinline__ float k916_f32(float x, float y, float erfcx_y, float sig1, const float *w) {
  const float h = 0.5f;
  const float ex2 = expf(-(x * x));
  const float xy = x * y;
  float s, c;
  sincosf(xy, &s, &c);
  const float sinc = (xy == 0.0f) ? 1.0f : __fdividef(s, xy);
  const float c2xy = c * c - s * s;
  // A fixed count of A916_TERMS_F32 terms from n0 (>= the window's
  // n1 - n0 + 1 for every x): every lane of a warp runs the same loop, and
  // the terms past n1 only widen the window.
  int n0, n1;
  a916_range_f32(x, n0, n1);
  const float nh0 = n0 * h;
  const float dm = nh0 - x;  // S3 offset: in [-4.3, 0.5]
  const float E3 = expf(-(dm * dm));
  const float rho3 = expf(-dm);  // in [0.6, 74]
  const float *wn = w + (n0 - 1);
  float acc3 = 0.0f, s23;
  // Beyond x = A916_TAIL_F32 - h every S2 term e^{-(nh+x)^2}, n >= 1, is
  // below e^{-18.49} (outside the window): when that holds for all the
  // warp's active lanes, the S2 series is left out (a warp-uniform choice,
  // so the lanes stay in lockstep).  Otherwise it runs over the first
  // A916_S2_TERMS_F32 terms; its offset is dp = nh0 + x = dm + 2x, so
  // rho2 = rho3 e^{-2x} and e^{-dp^2} = e^{-dm^2} (e^{-2x})^{2 n0 h}, taken
  // for n0 = 1 (every lane with x <= A916_TAIL_F32 - h); lanes with a
  // larger n0 leave S2 out, its terms being below e^{-18.49} there.
  if (__all_sync(__activemask(), x > A916_TAIL_F32 - h)) {
#pragma unroll
    for (int t = A916_TERMS_F32 - 1; t >= 0; --t) acc3 = fmaf(rho3, acc3, A916_GAUSS_F32[t] * wn[t]);
    s23 = E3 * acc3;
  } else {
    const float g = expf(-2.0f * x);
    const float rho2 = rho3 * g;  // e^{-dp}, below e^{-1/2}
    const float E2 = n0 == 1 ? E3 * g : 0.0f;
    float acc2 = 0.0f;
#pragma unroll
    for (int t = A916_TERMS_F32 - 1; t >= A916_S2_TERMS_F32; --t)
      acc3 = fmaf(rho3, acc3, A916_GAUSS_F32[t] * wn[t]);
#pragma unroll
    for (int t = A916_S2_TERMS_F32 - 1; t >= 0; --t) {
      const float ct = A916_GAUSS_F32[t] * wn[t];
      acc3 = fmaf(rho3, acc3, ct);
      acc2 = fmaf(rho2, acc2, ct);
    }
    s23 = fmaf(E2, acc2, E3 * acc3);
  }
  const float k2h = 0.31830988618f;  // 2h/pi
  float K = ex2 * erfcx_y * c2xy;
  K += k2h * x * ex2 * s * sinc;
  K += k2h * (0.5f * y * s23 - y * c2xy * ex2 * sig1);
  return K;
}

}  // namespace helk
