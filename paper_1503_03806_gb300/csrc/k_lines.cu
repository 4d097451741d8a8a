// k_lines.cu -- line-list kernels: validation, ordering by nu0, per-condition
// line preparation (Sec. 2.3-2.4) and the grid-tile -> line-range map.
//
// This translation unit is compiled with --fmad=false: the quantities that
// decide which grid points a line covers (window bounds) and which method
// evaluates a point (a, ku) must be the correctly rounded results of the
// operations written here, with no contraction into FMA.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "helk_internal.cuh"
#include "voigt_common.cuh"

namespace helk {

// e^{-(n h)^2}, h = 1/2, n = 1..13: weights of the S1 series of
// Algorithm 916 (depends on the line's damping only, so it is summed once
// per line).
__constant__ double c_exp_nh2[A916_S1_TERMS] = {
    0.77880078307140486825,  0.3678794411714423216,   0.10539922456186433678,
    0.018315638888734180294, 0.0019304541362277092422, 0.0001234098040866795495,
    4.7851173921290090896e-6, 1.1253517471925911451e-7, 1.6052280551856116087e-9,
    1.3887943864964020595e-11, 7.2877240958196924193e-14, 2.3195228302435693883e-16,
    4.477732441718301199e-19};

// -------------------------------------------------------- validation ---
__global__ void k_validate(int64_t n, const double *__restrict__ nu0, const double *__restrict__ S0,
                           const double *__restrict__ El, const double *__restrict__ gair,
                           const double *__restrict__ gself, const double *__restrict__ ncoll,
                           const double *__restrict__ delta, const double *__restrict__ lmass,
                           const double *__restrict__ lweight, DevStats *st) {
  int bad = 0, unsorted = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    double v = nu0[l];
    bool ok = isfinite(v) && v > 0.0 && isfinite(S0[l]) && S0[l] >= 0.0 && isfinite(gair[l]) &&
              gair[l] >= 0.0;
    if (El) ok = ok && isfinite(El[l]);
    if (gself) ok = ok && isfinite(gself[l]) && gself[l] >= 0.0;
    if (ncoll) ok = ok && isfinite(ncoll[l]);
    if (delta) ok = ok && isfinite(delta[l]);
    if (lmass) ok = ok && isfinite(lmass[l]) && lmass[l] > 0.0;
    if (lweight) ok = ok && isfinite(lweight[l]) && lweight[l] >= 0.0;
    bad += !ok;
    if (l + 1 < n && nu0[l + 1] < v) unsorted = 1;
  }
  if (bad) atomicAdd(&st->bad_lines, bad);
  if (unsorted) atomicOr(&st->unsorted, 1);
}

cudaError_t launch_validate_lines(helk_ctx *c, int64_t n) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > c->num_sms * 8) blocks = c->num_sms * 8;
  ++c->launches;
  k_validate<<<blocks, 256, 0, c->stream>>>(n, c->nu0, c->S0, c->has_E ? c->El : nullptr, c->gair,
                                            c->has_gself ? c->gself : nullptr,
                                            c->has_ncoll ? c->ncoll : nullptr,
                                            c->has_delta ? c->delta : nullptr,
                                            c->has_mass ? c->lmass : nullptr,
                                            c->has_weight ? c->lweight : nullptr, c->stats);
  return cudaGetLastError();
}

// ------------------------------------------- stable LSD radix sort (pairs) --
// Keys: 64-bit, values: 32-bit.  One pass per 8-bit digit; each pass is
// upsweep (per-tile digit counts) -> exclusive scan -> downsweep (stable
// scatter: warps own consecutive sub-ranges, ranks inside a warp batch come
// from the digit's peer lanes).
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_TILE = 4096;  // elements per block

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const unsigned long long *__restrict__ keys,
                                                           int64_t n, int shift, uint32_t *counts,
                                                           int nblk) {
  __shared__ uint32_t h[256];
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) h[d] = 0;
  __syncthreads();
  int64_t b0 = (int64_t)blockIdx.x * RS_TILE;
  int64_t b1 = b0 + RS_TILE < n ? b0 + RS_TILE : n;
  for (int64_t e = b0 + threadIdx.x; e < b1; e += RS_THREADS)
    atomicAdd(&h[(keys[e] >> shift) & 0xFF], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) counts[(int64_t)d * nblk + blockIdx.x] = h[d];
}

// Exclusive scan of m counts in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *counts, int64_t m) {
  __shared__ uint32_t wsum[32];
  int64_t per = (m + 1023) / 1024;
  int64_t s0 = threadIdx.x * per, s1 = s0 + per < m ? s0 + per : m;
  uint32_t s = 0;
  for (int64_t i = s0; i < s1; ++i) s += counts[i];
  // block exclusive scan of s
  uint32_t v = s;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    uint32_t x = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  uint32_t excl = v - s + (w > 0 ? wsum[w - 1] : 0u);
  for (int64_t i = s0; i < s1; ++i) {
    uint32_t t = counts[i];
    counts[i] = excl;
    excl += t;
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_downsweep(
    const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
    unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
    const uint32_t *__restrict__ counts, int nblk) {
  __shared__ uint32_t h[256 * RS_WARPS];  // [digit][warp]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 256 * RS_WARPS; i += RS_THREADS) h[i] = 0;
  __syncthreads();
  int64_t b0 = (int64_t)blockIdx.x * RS_TILE;
  int64_t b1 = b0 + RS_TILE < n ? b0 + RS_TILE : n;
  const int per = RS_TILE / RS_WARPS;
  int64_t w0 = b0 + (int64_t)w * per, w1 = w0 + per < b1 ? w0 + per : b1;
  // per-warp digit counts
  for (int64_t e0 = w0; e0 < w1; e0 += 32) {
    int64_t e = e0 + lane;
    const bool valid = e < w1;
    uint32_t d = valid ? (uint32_t)((kin[e] >> shift) & 0xFF) : 0u;
    uint32_t peers = warp_digit_peers(d, valid);
    if (valid && (peers & lanemask_lt()) == 0) h[d * RS_WARPS + w] += __popc(peers);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    uint32_t run = counts[(int64_t)d * nblk + blockIdx.x];
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      uint32_t t = h[d * RS_WARPS + ww];
      h[d * RS_WARPS + ww] = run;
      run += t;
    }
  }
  __syncthreads();
  for (int64_t e0 = w0; e0 < w1; e0 += 32) {
    int64_t e = e0 + lane;
    bool valid = e < w1;
    unsigned long long k = valid ? kin[e] : 0ull;
    uint32_t d = valid ? (uint32_t)((k >> shift) & 0xFF) : 0u;
    uint32_t peers = warp_digit_peers(d, valid);
    if (valid) {
      uint32_t pos = h[d * RS_WARPS + w] + __popc(peers & lanemask_lt());
      kout[pos] = k;
      vout[pos] = vin[e];
    }
    __syncwarp();
    if (valid && (peers & lanemask_lt()) == 0) h[d * RS_WARPS + w] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_line_keys(int64_t n, const double *__restrict__ nu0, unsigned long long *keys,
                            uint32_t *vals) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    double v = nu0[l];
    if (v == 0.0) v = 0.0;  // -0 -> +0
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    keys[l] = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    vals[l] = (uint32_t)l;
  }
}

__global__ void k_gather(int64_t n, const uint32_t *__restrict__ perm, const double *__restrict__ src,
                         double *__restrict__ dst) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    dst[l] = src[perm[l]];
}

cudaError_t launch_sort_lines(helk_ctx *c, int64_t n) {
  if (n <= 1) return cudaSuccess;
  const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
  // scratch: 2 key arrays, 2 value arrays, counts, one double array
  int64_t need = 2 * n * 8 + 2 * n * 4 + (int64_t)256 * nblk * 4 + n * 8 + 64;
  helk_status st = ensure_buf(c, &c->tmp, &c->tmp_cap, need, "line sort scratch");
  if (st != HELK_OK) return cudaErrorMemoryAllocation;
  char *p = (char *)c->tmp;
  unsigned long long *ka = (unsigned long long *)p;  p += n * 8;
  unsigned long long *kb = (unsigned long long *)p;  p += n * 8;
  uint32_t *va = (uint32_t *)p;                      p += n * 4;
  uint32_t *vb = (uint32_t *)p;                      p += n * 4;
  uint32_t *counts = (uint32_t *)p;                  p += (int64_t)256 * nblk * 4;
  p = (char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  double *dtmp = (double *)p;
  int gb = (int)((n + 255) / 256);
  if (gb > c->num_sms * 16) gb = c->num_sms * 16;
  ++c->launches;
  k_line_keys<<<gb, 256, 0, c->stream>>>(n, c->nu0, ka, va);
  for (int pass = 0; pass < 8; ++pass) {
    int shift = pass * 8;
    ++c->launches;
    k_rs_upsweep<<<nblk, RS_THREADS, 0, c->stream>>>(ka, n, shift, counts, nblk);
    ++c->launches;
    k_rs_scan<<<1, 1024, 0, c->stream>>>(counts, (int64_t)256 * nblk);
    ++c->launches;
    k_rs_downsweep<<<nblk, RS_THREADS, 0, c->stream>>>(ka, va, kb, vb, n, shift, counts, nblk);
    unsigned long long *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  double *fields[9] = {c->nu0, c->S0, c->has_E ? c->El : nullptr, c->gair,
                       c->has_gself ? c->gself : nullptr, c->has_ncoll ? c->ncoll : nullptr,
                       c->has_delta ? c->delta : nullptr, c->has_mass ? c->lmass : nullptr,
                       c->has_weight ? c->lweight : nullptr};
  for (int f = 0; f < 9; ++f) {
    if (!fields[f]) continue;
    ++c->launches;
    k_gather<<<gb, 256, 0, c->stream>>>(n, va, fields[f], dtmp);
    cudaError_t e = cudaMemcpyAsync(fields[f], dtmp, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------- line preparation --
struct PrepArgs {
  double mass;
  int cut_kind;
  double cut_value, cut_cap;
  double nu_min, dnu;
  int64_t ngrid;
};

// Per line and condition, in the operation order of the definitions:
//   nu0' = nu0 + delta P                                   (Sec. 2.3 shift)
//   S    = S0 (Q0/Q) e^{-c2E/T + c2E/T0} (1-e^{-c2 nu0/T})/(1-e^{-c2 nu0/T0})
//   S   *= abundance weight of the line's species          (Sec. 2.1)
//   Gamma_L = (T0/T)^n (g_air (P - P/2) + g_self P/2)      (Sec. 2.3)
//   Gamma_D = nu0' sqrt(2 ln2 k_B T / m) / c               (Sec. 2.3)
//   a = sqrt(ln2) Gamma_L / Gamma_D, ku = sqrt(ln2)/Gamma_D,
//   S' = S sqrt(ln2/pi) / Gamma_D, window from the cutoff   (Sec. 2.4)
// blockIdx.y is the condition; records of condition k start at k * n.
__global__ void k_lineprep(int64_t n, const double *__restrict__ nu0, const double *__restrict__ S0,
                           const double *__restrict__ El, const double *__restrict__ gair,
                           const double *__restrict__ gself, const double *__restrict__ ncoll,
                           const double *__restrict__ delta, const double *__restrict__ lmass,
                           const double *__restrict__ lweight, PrepArgs A,
                           const CondArgs *__restrict__ conds, CondArgs single,
                           LineRec64 *__restrict__ rec_all, double *__restrict__ ckey,
                           CondStats *cst_all, int a916_f64) {
  const int cond = blockIdx.y;
  const CondArgs C = conds ? conds[cond] : single;
  LineRec64 *rec = rec_all + (int64_t)cond * n;
  CondStats *cst = cst_all + cond;
  unsigned long long evals = 0;
  long long wmax = -1;
  unsigned long long spmax = 0;
  const double vth = sqrt(2.0 * LN2 * KB * C.T / (A.mass * AMU)) / CLIGHT;
  const double tfac_half = sqrt(T0 / C.T);  // (T0/T)^n for the usual n = 1/2
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    const double v0 = nu0[l];
    const double dl = delta ? delta[l] : 0.0;
    const double ga = gair[l];
    const double gs = gself ? gself[l] : ga;
    const double nc = ncoll ? ncoll[l] : 0.5;
    double S = S0[l];
    const double nu0p = v0 + dl * C.P;
    if (El) {
      const double E = El[l];
      const double boltz = exp(-C2 * E / C.T + C2 * E / T0);
      const double stim = v0 > 0.0 ? expm1(-C2 * v0 / C.T) / expm1(-C2 * v0 / T0) : T0 / C.T;
      S = S * C.q_ratio * boltz * stim;
    }
    if (lweight) S = S * lweight[l];
    const double tfac = (nc == 0.5) ? tfac_half : pow(T0 / C.T, nc);
    const double pself = 0.5 * C.P;
    const double gL = tfac * (ga * (C.P - pself) + gs * pself);
    const double gD = nu0p * (lmass ? sqrt(2.0 * LN2 * KB * C.T / (lmass[l] * AMU)) / CLIGHT : vth);
    // The FP64 form divides (a and k_u are then the correctly rounded results
    // the oracle computes, so every method choice matches it); the FP32 form
    // rounds them to FP32 anyway and multiplies by one reciprocal (FP64
    // divisions are long sequences on the scarce FP64 unit).
    double a, ku, Sp;
    if (a916_f64) {
      a = SQRTLN2 * gL / gD;
      ku = SQRTLN2 / gD;
      Sp = S * SQRTLN2PI / gD;
    } else {
      const double igD = 1.0 / gD;
      a = SQRTLN2 * gL * igD;
      ku = SQRTLN2 * igD;
      Sp = S * SQRTLN2PI * igD;
    }
    double cut;
    if (A.cut_kind == HELK_CUT_ABS) cut = A.cut_value;
    else if (A.cut_kind == HELK_CUT_LORENTZ) cut = fmin(A.cut_value * gL, A.cut_cap);
    else cut = INFINITY;
    double lo, hi;
    if (A.cut_kind == HELK_CUT_NONE) {
      lo = 0.0;
      hi = (double)(A.ngrid - 1);
    } else {
      lo = ceil((nu0p - cut - A.nu_min) / A.dnu);
      hi = floor((nu0p + cut - A.nu_min) / A.dnu);
      if (lo < 0.0) lo = 0.0;
      if (hi > (double)(A.ngrid - 1)) hi = (double)(A.ngrid - 1);
      if (lo > (double)A.ngrid) lo = (double)A.ngrid;
      if (hi < -1.0) hi = -1.0;
    }
    LineRec64 r;
    r.nu0p = nu0p;
    r.ku = ku;
    r.a = a;
    r.a2 = a * a;
    r.Sp = Sp;
    r.ilo = (int32_t)lo;
    r.ihi = (int32_t)hi;
    // Algorithm 916 per-line factors (only reachable when a < 10); the FP32
    // form takes them in FP32 when packing its records
    if (a916_f64 && a < 10.0) {
      r.erfcx_a = erfcx(a);
      double s1 = 0.0;
      for (int k = 0; k < A916_S1_TERMS; ++k) {
        double nh = (double)(k + 1) * A916_H;
        s1 += c_exp_nh2[k] / (nh * nh + a * a);
      }
      r.sig1 = s1;
    } else {
      r.erfcx_a = 0.0;
      r.sig1 = 0.0;
    }
    rec[l] = r;
    // reference index of the unshifted centre: non-decreasing in list order
    double ck = floor((v0 - A.nu_min) / A.dnu);
    if (ck < -4.0e15) ck = -4.0e15;
    if (ck > 4.0e15) ck = 4.0e15;
    if (cond == 0) ckey[l] = ck;
    if (r.ihi >= r.ilo) {
      evals += (unsigned long long)(r.ihi - r.ilo + 1);
      long long c0 = (long long)ck;
      long long h1 = c0 - r.ilo, h2 = (long long)r.ihi - c0;
      long long hw = h1 > h2 ? h1 : h2;
      if (hw > wmax) wmax = hw;
      unsigned long long sb = (unsigned long long)__double_as_longlong(Sp);
      if (sb > spmax) spmax = sb;
    }
  }
  // warp-aggregate then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_down_sync(0xffffffffu, evals, o);
    long long w2 = __shfl_down_sync(0xffffffffu, wmax, o);
    if (w2 > wmax) wmax = w2;
    unsigned long long s2 = __shfl_down_sync(0xffffffffu, spmax, o);
    if (s2 > spmax) spmax = s2;
  }
  if ((threadIdx.x & 31) == 0) {
    if (evals) atomicAdd(&cst->evals, evals);
    if (wmax >= 0) atomicMax(&cst->wmax, wmax);
    if (spmax) atomicMax(&cst->spmax_bits, spmax);
  }
}

static int line_blocks(helk_ctx *c, int64_t n, int n_cond) {
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = std::max<int64_t>(1, (int64_t)c->num_sms * 16 / std::max(1, n_cond));
  if (blocks > cap) blocks = cap;
  return (int)std::max<int64_t>(1, blocks);
}

cudaError_t launch_lineprep(helk_ctx *c, int n_cond, const CondArgs *single, double mass,
                            const helk_cutoff &cut, const helk_grid &g, bool a916_f64) {
  const int64_t n = c->nlines;
  if (n <= 0) return cudaSuccess;
  PrepArgs A{mass, cut.kind, cut.value, cut.cap, g.nu_min, g.dnu, g.n};
  const CondArgs one = single ? *single : CondArgs{0, 0, 0, 0};
  dim3 grid(line_blocks(c, n, n_cond), n_cond);
  ++c->launches;
  k_lineprep<<<grid, 256, 0, c->stream>>>(
      n, c->nu0, c->S0, c->has_E ? c->El : nullptr, c->gair, c->has_gself ? c->gself : nullptr,
      c->has_ncoll ? c->ncoll : nullptr, c->has_delta ? c->delta : nullptr,
      c->has_mass ? c->lmass : nullptr, c->has_weight ? c->lweight : nullptr, A,
      single ? nullptr : c->cond_dev, one, c->rec64, c->ckey, c->cstats, a916_f64 ? 1 : 0);
  return cudaGetLastError();
}

// ----------------------------------------------------- FP32 line records --
// From the FP64 records: strengths scaled by 2^-E (E from the largest S' of
// the condition, so every scaled term is <= 1 and the FP32 range covers 38
// decades below it); the centre as the integer grid index c plus the FP32
// offset phi = (nu0' - nu_c) ku, so that u_i = (i - c) beta - phi keeps full
// relative precision near the line centre.
// the 3-node GH factor over S' a: (sqrt(pi)/6)/pi, as one constant (one FP64
// multiplication a line instead of a division)
constexpr double P3_FACTOR = SQRTPI / 6.0 / PI;

__global__ void k_pack32(int64_t n, const LineRec64 *__restrict__ r64_all, double nu_min, double dnu, int64_t ngrid,
                         const double *__restrict__ ckey, CondStats *cst_all, LineRec32 *__restrict__ r32_all,
                         int2 *__restrict__ core_all, int32_t *__restrict__ ckey32, int *err_flags,
                         int *__restrict__ core_blk_all, int nblk) {
  const int cond = blockIdx.y;
  const LineRec64 *r64 = r64_all + (int64_t)cond * n;
  LineRec32 *r32 = r32_all + (int64_t)cond * n;
  CondStats *cst = cst_all + cond;
  const double spmax = __longlong_as_double((long long)cst->spmax_bits);
  const int E = spmax > 0.0 ? ilogb(spmax) + 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) cst->scale_exp = E;
  const double pow2mE = ldexp(1.0, -E);  // exact: S' 2^-E by one multiplication
  const double idnu = 1.0 / dnu;
  int cw1 = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    const LineRec64 r = r64[l];
    // the reference index is an integer below 2^53 in magnitude: integer
    // operations from here on (the FP64 unit bounds this kernel)
    const long long key = (long long)ckey[l];
    const int k32 = (int)min(max(key, -2147483647ll), 2147483647ll);
    if (cond == 0) ckey32[l] = k32;
    LineRec32 q;
    // any integer within a step of the centre serves as c (phi takes the
    // rest), so a product by 1/dnu replaces the division
    // (clamped to the grid, [0, ngrid - 1]: exact for every centre on the
    // grid, and i - c then fits in 32 bits for every grid index i; a centre
    // off the grid leaves its offset in phi, which has the sign of i - c, so
    // u = (i - c) beta - phi takes no cancellation)
    double cf = rint((r.nu0p - nu_min) * idnu);
    const bool clamped = cf < 0.0 || cf > (double)(ngrid - 1);
    if (cf < 0.0) cf = 0.0;
    if (cf > (double)(ngrid - 1)) cf = (double)(ngrid - 1);
    q.c = (int32_t)cf;
    q.ilo = r.ilo;
    q.ihi = r.ihi;
    q.phi_k = (float)((r.nu0p - (nu_min + cf * dnu)) * r.ku);
    q.beta = (float)(dnu * r.ku);
    q.a = (float)r.a;
    q.a2 = (float)r.a2;
    const double sp = r.Sp * pow2mE;
    q.P1 = (float)(sp * r.a * INV_SQRTPI);
    q.P3 = (float)(sp * r.a * P3_FACTOR);
    q.Sp = (float)sp;
    if (q.a < 10.0f) {  // Algorithm 916 per-line factors, in FP32
      q.erfcx_a = erfcxf(q.a);
      float s1 = 0.0f;
      for (int k = 0; k < A916_S1_TERMS; ++k) {
        const float nh = (float)(k + 1) * (float)A916_H;
        s1 += (float)c_exp_nh2[k] / (nh * nh + q.a2);
      }
      q.sig1 = s1;
    } else {
      q.erfcx_a = 0.0f;
      q.sig1 = 0.0f;
    }
    r32[l] = q;
    // The line's core in the FP32 arithmetic of the Voigt kernels: points with
    // fma(u, u, a^2) < 100, u = fma(i - c, beta, -phi), so |u| < 10.  With the
    // centre on the grid (|phi| <= beta/2) that needs |i - c| <= (10 + |phi|)/beta.
    // With a centre off the grid, c clamped to the nearer end, phi has the
    // sign of i - c, so |u| = |i - c| beta + |phi| and the core needs
    // |i - c| < (10 - |phi|)/beta: none once |phi| >= 10.  The farthest core
    // point from the reference index bounds the core kernel's candidate
    // search.
    int2 core = make_int2(1, 0);
    int line_w1 = 0;  // 1 + the line's core reach, 0: no core
    if (q.a2 < 100.0f && q.ihi >= q.ilo && q.beta > 0.0f) {
      const float reach = clamped ? 10.001f - fabsf(q.phi_k) : 10.001f + fabsf(q.phi_k);
      if (reach > 0.0f) {
        // an upper bound (FP32 quotient, rounding covered by the margin of 2)
        const float dmaxf = ceilf(reach / q.beta) + 2.0f;
        // Both Voigt kernels take i - c exactly in FP32 only within 2^24
        // points of c, so a core must end within 2^23 points (beta above
        // ~1.2e-6: a Doppler width below ~7e5 grid steps); else the call is
        // reported as unsupported by the FP32 form.
        if (dmaxf >= 8388608.0f) atomicOr(err_flags, ERRF_F32_RANGE);
        const long long dmax = (long long)fminf(dmaxf, 4.0e9f);
        const long long clo = max((long long)q.ilo, (long long)q.c - dmax);
        const long long chi = min((long long)q.ihi, (long long)q.c + dmax);
        if (clo <= chi) {
          const long long w = max(key - clo, chi - key);
          line_w1 = (int)min(w + 1, 2000000000ll);
          cw1 = max(cw1, line_w1);
          core = make_int2((int)clo, (int)chi);
        }
      }
    }
    core_all[(int64_t)cond * n + l] = core;
    // The reach of the lines whose reference index lies in each block of
    // CORE_BLK_PTS grid points (the core kernel's candidate window): the
    // list is ordered by the index, so the lanes of a warp mostly share a
    // block and one atomic per block and warp suffices.
    const int blk = min(max(k32 >> 12, 0), nblk - 1);  // CORE_BLK_PTS = 2^12
    const unsigned peers = __match_any_sync(__activemask(), blk);
    const int wblk = __reduce_max_sync(peers, line_w1);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && wblk > 0)
      atomicMax(&core_blk_all[(int64_t)cond * nblk + blk], wblk);
  }
  for (int o = 16; o > 0; o >>= 1) cw1 = max(cw1, __shfl_down_sync(0xffffffffu, cw1, o));
  if ((threadIdx.x & 31) == 0 && cw1 > 0) atomicMax(&cst->core_w1, cw1);
}

cudaError_t launch_pack32(helk_ctx *c, int n_cond, const helk_grid &g) {
  const int64_t n = c->nlines;
  if (n <= 0) return cudaSuccess;
  dim3 grid(line_blocks(c, n, n_cond), n_cond);
  ++c->launches;
  k_pack32<<<grid, 256, 0, c->stream>>>(n, c->rec64, g.nu_min, g.dnu, g.n, c->ckey, c->cstats, c->rec32,
                                        c->core_rng, c->ckey32, &c->stats->err_flags, c->core_blk,
                                        core_blocks(g.n));
  return cudaGetLastError();
}

// --------------------------------------------------------------- tile map --
// Lines overlapping grid tile [A, B) have their reference index in
// [A - W, B - 1 + W], W = max half-width of any window of the condition: a
// contiguous range of the nu0-ordered list, found by two searches.  One warp
// per tile searches 32-ary: each step the lanes probe 32 evenly spaced keys
// and a ballot narrows the range 32-fold (5 dependent loads for 1e6 lines
// instead of 20 for a binary search).

__global__ void k_tilemap(int64_t nlines, const double *__restrict__ ckey, int64_t ngrid, int tile,
                          int64_t ntiles, const CondStats *__restrict__ cst, int32_t *tlo,
                          int32_t *thi) {
  const int cond = blockIdx.y;
  const int64_t t = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  if (t >= ntiles) return;  // warp-uniform
  const int64_t o = (int64_t)cond * ntiles + t;
  const long long W = cst[cond].wmax;
  const int lane = threadIdx.x & 31;
  if (W < 0) {  // no line has a non-empty window
    if (lane == 0) tlo[o] = thi[o] = 0;
    return;
  }
  const double A = (double)(t * tile);
  const double B = (double)((t + 1) * tile < ngrid ? (t + 1) * tile : ngrid);
  const double klo = A - (double)W, khi = B - 1.0 + (double)W;
  const int64_t first = warp_search(ckey, 0, nlines, klo, false);  // first key >= klo
  const int64_t last = warp_search(ckey, first, nlines, khi, true); // first key > khi
  if (lane == 0) {
    tlo[o] = (int32_t)first;
    thi[o] = (int32_t)last;
  }
}

cudaError_t launch_tilemap(helk_ctx *c, int n_cond, const helk_grid &g, int tile, int64_t ntiles) {
  dim3 grid((unsigned)((ntiles + 7) / 8), n_cond);  // 8 warps, one tile each
  ++c->launches;
  k_tilemap<<<grid, 256, 0, c->stream>>>(c->nlines, c->ckey, g.n, tile, ntiles, c->cstats,
                                         c->tile_lo, c->tile_hi);
  return cudaGetLastError();
}

// ------------------------------------------------------- condition order --
// Largest evaluation count first, so the persistent Voigt kernel's last
// items are the cheapest (ties keep the input order).
__global__ void k_cond_order(int n_cond, const CondStats *__restrict__ cst, int *order) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < n_cond; ++i) {
    const unsigned long long e = cst[i].evals;
    int j = i;
    while (j > 0 && cst[order[j - 1]].evals < e) {
      order[j] = order[j - 1];
      --j;
    }
    order[j] = i;
  }
}

cudaError_t launch_cond_order(helk_ctx *c, int n_cond) {
  ++c->launches;
  k_cond_order<<<1, 32, 0, c->stream>>>(n_cond, c->cstats, c->cond_order);
  return cudaGetLastError();
}

}  // namespace helk
