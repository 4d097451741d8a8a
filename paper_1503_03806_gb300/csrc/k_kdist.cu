// k_kdist.cu -- k-distribution tables (Sec. 2.2, 2.6).
//
// One CTA per bin: the bin's opacities (non-negative doubles, ordered as
// their IEEE bit patterns) are radix-sorted in shared memory when they fit
// (else in a global ping-pong buffer), then the same CTA computes
// L_j = ln max(k_j, kappa_floor) on g_j = (j + 1/2)/N_b and the least-squares
// Chebyshev coefficients c = P L, where P is the pseudo-inverse of the design
// matrix (shared by all bins of one size; computed once by k_pinv).
//
// FP64 is the scarce unit of this GPU (1/64 of the FP32 rate), so the two
// per-point costs that would be FP64 are moved to FP32 where that keeps
// FP64-level accuracy: ln takes its second-order tail in FP32 (absolute
// error < 1e-13), and c = P L is a double-float dot product -- P and L are
// each split into FP32 high and low parts, and every term hi*hi is summed
// exactly (two-product and two-sum), the cross terms in FP32 (relative
// error ~2^-46 of the sum of |P_kj L_j|).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "helk_internal.cuh"

namespace helk {

constexpr int KD_THREADS = 512;
constexpr int KD_WARPS = KD_THREADS / 32;
constexpr int NCHEB_MAX = 32;
constexpr int KD_LNTAB = 256;  // float2 entries: ln c_j, then 1/c_j

__device__ __forceinline__ uint32_t lanemask_lt_kd() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- logarithm --
// ln x for a positive double by the table-driven method of Tang (ACM TOMS
// 16(4), 1990): x = 2^e m with m in [1, 2), c_j = 1 + j/128 where j is the
// top 7 fraction bits of m, so f = m - c_j is exact and r = f / c_j lies in
// [0, 1/128); then ln x = e ln2 + ln c_j + log1p(r), with log1p(r) to r^7
// (truncation < 2^-59).  The 128 entries ln c_j, 1/c_j live in shared memory.
// It is computed as an FP32 (high, low) pair with integer and FP32
// operations only (FP64 runs at 1/64 of the FP32 rate here).  From the
// key bits: e, j and f = F 2^-52 with F the 45 fraction bits below j, split
// exactly into two floats; r = f (1/c_j) in float-float (1/c_j as a pair);
// ln x = e ln2 + ln c_j + r - r^2/2 + r^3 q(r), the large terms added by
// two-sum, ln2 in three parts (the first with 12 bits, so e * ln2_hi is
// exact), the cubic remainder (< 2^-21) in plain FP32.  Absolute error
// < 2e-12 for |ln x| < 70, < 2e-11 over the normal range (float-float
// resolution of |ln x|).
constexpr float LN2_HI_F = 0x1.62ep-1f;      // 2839/4096
constexpr float LN2_MID_F = 0x1.0bfbe8p-15f;
constexpr float LN2_LO_F = 0x1.cf78p-40f;

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ float2 log_ff(unsigned long long b, const float2 *lnc, const float2 *invc) {
  const int ex = (int)(b >> 52);
  if (ex == 0) {  // subnormal: the library log, then split
    const double L = log(__longlong_as_double((long long)b));
    const float hi = (float)L;
    return make_float2(hi, (float)(L - (double)hi));
  }
  const int j = (int)((b >> 45) & 0x7F);
  const unsigned long long F = b & 0x1FFFFFFFFFFFull;
  const float fh = (float)(unsigned)(F >> 21) * 0x1p-31f;        // top 24 bits, exact
  const float fl = (float)(unsigned)(F & 0x1FFFFFu) * 0x1p-52f;  // low 21 bits, exact
  const float2 ic = invc[j];
  float rh = fh * ic.x;
  float rl = fmaf(fh, ic.x, -rh);
  rl = fmaf(fh, ic.y, rl);
  rl = fmaf(fl, ic.x, rl);
  {
    const float t = rh + rl;  // |rh| >= |rl|
    rl = rl - (t - rh);
    rh = t;
  }
  const float p = rh * rh;
  float pe = fmaf(rh, rh, -p);
  pe = fmaf(2.0f * rh, rl, pe);
  float q = fmaf(rh, 1.0f / 7.0f, -1.0f / 6.0f);
  q = fmaf(q, rh, 1.0f / 5.0f);
  q = fmaf(q, rh, -1.0f / 4.0f);
  q = fmaf(q, rh, 1.0f / 3.0f);
  const float cub = (rh * rh) * (rh * q);
  const float2 lc = lnc[j];
  const float ef = (float)(ex - 1023);
  const float mh = ef * LN2_MID_F;
  const float ml = fmaf(ef, LN2_MID_F, -mh);
  float s, e1, e2, e3, e4;
  two_sum_f(ef * LN2_HI_F, lc.x, s, e1);
  two_sum_f(s, mh, s, e2);
  two_sum_f(s, rh, s, e3);
  two_sum_f(s, -0.5f * p, s, e4);
  float lo = ((e1 + e2) + (e3 + e4)) + (lc.y + ml);
  lo = fmaf(ef, LN2_LO_F, lo);
  lo = fmaf(-0.5f, pe, lo + rl) + cub;
  const float hi = s + lo;
  return make_float2(hi, lo - (hi - s));
}

// ------------------------------------------------------ pseudo-inverse --
// Position of P[k][j] (j < ceil(N_b/2)) in the blocked layout of the
// symmetrized half: blocks of 32 columns, each [k][32].
__host__ __device__ __forceinline__ int64_t pinv_index(int k, int64_t j, int ncheb) {
  return ((j >> 5) * ncheb + k) * 32 + (j & 31);
}
constexpr int PINV_MIN_COLS = 64;  // buffers hold max(N_b, 64) columns
// The design matrix A_jk = T_k(t_j), t_j = (2j+1)/N_b - 1, is the same for
// every bin, so its pseudo-inverse P = R^{-1} Q_1^T (Householder QR, A = QR)
// is computed once per (N_b, n_cheb) and each bin's coefficients are
// c = P L.  One CTA; A is built column-major in `work` (n_cheb columns of
// N_b), Q_1 is formed in `P` and turned into P column by column.
constexpr int PI_THREADS = 512;

__device__ double block_sum_pi(double v, double *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < PI_THREADS / 32; ++i) s += red[i];
  return s;
}

// `tag` (optional, device): the (N_b, n_cheb) whose pseudo-inverse P
// already holds; the kernel returns at once when they equal this call's and
// records them when it has rebuilt P.
__global__ void __launch_bounds__(PI_THREADS) k_pinv(int64_t nb, int ncheb, double *work,
                                                     double *vtv_out, double *P, float2 *lntab,
                                                     long long *tag) {
  __shared__ double red[PI_THREADS / 32];
  __shared__ double R[NCHEB_MAX * NCHEB_MAX];
  __shared__ double vtv[NCHEB_MAX];
  __shared__ int s_current;
  const int tid = threadIdx.x;
  if (tag) {
    if (tid == 0) s_current = tag[0] == (long long)nb && tag[1] == (long long)ncheb;
    __syncthreads();
    if (s_current) return;
  }
  // A, column-major
  for (int64_t j = tid; j < nb; j += PI_THREADS) {
    const double t = (double)(2 * j + 1) / (double)nb - 1.0;
    double tkm1 = 1.0, tk = t;
    work[j] = 1.0;
    if (ncheb > 1) work[nb + j] = t;
    for (int k = 2; k < ncheb; ++k) {
      const double tn = 2.0 * t * tk - tkm1;
      tkm1 = tk;
      tk = tn;
      work[(int64_t)k * nb + j] = tn;
    }
  }
  __syncthreads();
  // Householder QR: column c becomes the reflector v_c (rows c..nb-1)
  for (int c = 0; c < ncheb; ++c) {
    double *col = work + (int64_t)c * nb;
    double s = 0.0;
    for (int64_t j = c + tid; j < nb; j += PI_THREADS) s += col[j] * col[j];
    const double norm = sqrt(block_sum_pi(s, red));
    const double x0 = col[c];
    const double alpha = x0 > 0.0 ? -norm : norm;
    __syncthreads();
    if (tid == 0) col[c] = x0 - alpha;
    __syncthreads();
    s = 0.0;
    for (int64_t j = c + tid; j < nb; j += PI_THREADS) s += col[j] * col[j];
    const double vv = block_sum_pi(s, red);
    if (tid == 0) {
      vtv[c] = vv;
      R[c * NCHEB_MAX + c] = alpha;
    }
    for (int cc = c + 1; cc < ncheb; ++cc) {
      double *oc = work + (int64_t)cc * nb;
      s = 0.0;
      for (int64_t j = c + tid; j < nb; j += PI_THREADS) s += col[j] * oc[j];
      const double f = 2.0 * block_sum_pi(s, red) / vv;
      for (int64_t j = c + tid; j < nb; j += PI_THREADS) oc[j] -= f * col[j];
      __syncthreads();
      if (tid == 0) R[c * NCHEB_MAX + cc] = oc[c];
    }
    __syncthreads();
  }
  // Q_1 = H_0 H_1 ... H_{n-1} [I; 0], column-major in P
  for (int k = 0; k < ncheb; ++k)
    for (int64_t j = tid; j < nb; j += PI_THREADS) P[(int64_t)k * nb + j] = (j == k) ? 1.0 : 0.0;
  __syncthreads();
  for (int c = ncheb - 1; c >= 0; --c) {
    const double *v = work + (int64_t)c * nb;
    for (int k = 0; k < ncheb; ++k) {
      double *e = P + (int64_t)k * nb;
      double s = 0.0;
      for (int64_t j = c + tid; j < nb; j += PI_THREADS) s += v[j] * e[j];
      const double f = 2.0 * block_sum_pi(s, red) / vtv[c];
      for (int64_t j = c + tid; j < nb; j += PI_THREADS) e[j] -= f * v[j];
      __syncthreads();
    }
  }
  // P[:, j] = R^{-1} Q_1[j, :]^T, k-major (P[k*nb + j])
  for (int64_t j = tid; j < nb; j += PI_THREADS) {
    double p[NCHEB_MAX];
    for (int k = ncheb - 1; k >= 0; --k) {
      double v = P[(int64_t)k * nb + j];
      for (int m = k + 1; m < ncheb; ++m) v -= R[k * NCHEB_MAX + m] * p[m];
      p[k] = v / R[k * NCHEB_MAX + k];
    }
    for (int k = 0; k < ncheb; ++k) P[(int64_t)k * nb + j] = p[k];
  }
  __syncthreads();
  // The abscissae are symmetric, t_{nb-1-j} = -t_j, and T_k(-t) = (-1)^k T_k(t),
  // so P[k][nb-1-j] = (-1)^k P[k][j]: only the symmetrized first half,
  // j < nh = ceil(nb/2), is kept, as FP32 (high, low) pairs in blocks of 32
  // columns, [j / 32][k][j % 32] (pinv_index; columns past nh are zero), so
  // that any run of whole blocks is one contiguous copy; built in `work` and
  // then moved to the front of P.
  const int64_t nh = (nb + 1) / 2;
  const int64_t npad = ((nh + 31) / 32) * 32;
  float2 *W = reinterpret_cast<float2 *>(work);
  for (int64_t e = tid; e < (int64_t)ncheb * npad; e += PI_THREADS) {
    const int k = (int)(e / npad);
    const int64_t j = e % npad;
    float2 v2 = make_float2(0.0f, 0.0f);
    if (j < nh) {
      const double v =
          0.5 * (P[(int64_t)k * nb + j] + ((k & 1) ? -1.0 : 1.0) * P[(int64_t)k * nb + (nb - 1 - j)]);
      const float hi = (float)v;
      v2 = make_float2(hi, (float)(v - (double)hi));
    }
    W[pinv_index(k, j, ncheb)] = v2;
  }
  __syncthreads();
  float2 *Ps = reinterpret_cast<float2 *>(P);
  for (int64_t e = tid; e < (int64_t)ncheb * npad; e += PI_THREADS) Ps[e] = W[e];
  if (tid == 0 && vtv_out) vtv_out[0] = vtv[0];
  // the logarithm's table, ln c_j and 1/c_j (c_j = 1 + j/128) as FP32
  // (high, low) pairs, computed here once instead of in every bin's CTA
  if (tid < 128) {
    const double cj = 1.0 + tid / 128.0, l = log(cj), ic = 1.0 / cj;
    const float lh = (float)l, ih = (float)ic;
    lntab[tid] = make_float2(lh, (float)(l - (double)lh));
    lntab[128 + tid] = make_float2(ih, (float)(ic - (double)ih));
  }
  if (tid == 0 && tag) {  // read by later launches only (stream order)
    tag[0] = (long long)nb;
    tag[1] = (long long)ncheb;
  }
}

// The pseudo-inverse buffer: max(nb, 64) ncheb doubles of work space (the
// blocked symmetrized half of P at its front when done; it takes at most
// ncheb (ceil(nb/2) + 31) FP32 pairs), then the logarithm's table.  The
// Householder work array k_pinv is given has the same size.
int64_t pinv_work_doubles(int64_t nb, int ncheb) { return std::max<int64_t>(nb, PINV_MIN_COLS) * ncheb; }
int64_t pinv_bytes(int64_t nb, int ncheb) { return (pinv_work_doubles(nb, ncheb) + KD_LNTAB) * 8; }

static float2 *pinv_lntab(helk_ctx *c, int64_t nb, int ncheb) {
  return reinterpret_cast<float2 *>(c->pinv + pinv_work_doubles(nb, ncheb));
}

cudaError_t launch_pinv(helk_ctx *c, int64_t nb, int ncheb, double *work) {
  ++c->launches;
  k_pinv<<<1, PI_THREADS, 0, c->stream>>>(nb, ncheb, work, nullptr, c->pinv, pinv_lntab(c, nb, ncheb),
                                        nullptr);
  return cudaGetLastError();
}

// --------------------------------------------------- block-wide helpers --
// Per-(digit, warp) counters, digit-major in scan order (position 16 d + w)
// but stored with row stride 17: the lanes of a warp look up counters of
// different digits, which stride 16 would put in 2 of the 32 banks.
constexpr int KD_HIST = 256 * (KD_WARPS + 1);
static_assert(KD_WARPS == 16, "counter layout assumes 16 warps");
__device__ __forceinline__ int hidx(uint32_t d, int w) { return (int)d * (KD_WARPS + 1) + w; }

// Exclusive scan of the KD_THREADS*8 counters in scan order, in place.
__device__ void block_exscan_4096(uint32_t *h, uint32_t *wtot) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t loc[8];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int pos = tid * 8 + i;
    loc[i] = h[pos + (pos >> 4)];
    s += loc[i];
  }
  uint32_t v = s;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wtot[w] = v;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < KD_WARPS ? wtot[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane < KD_WARPS) wtot[lane] = x;
  }
  __syncthreads();
  uint32_t run = v - s + (w > 0 ? wtot[w - 1] : 0u);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int pos = tid * 8 + i;
    h[pos + (pos >> 4)] = run;
    run += loc[i];
  }
  __syncthreads();
}

// Stable LSD radix sort of nb 64-bit keys held in A (shared or global);
// B is the second buffer.  Digits whose value is the same in every key are
// skipped.  Returns the buffer holding the result.
__device__ unsigned long long *cta_radix_sort(unsigned long long *A, unsigned long long *B, int nb,
                                              uint32_t *hist /* KD_HIST counters */, uint32_t *wtot,
                                              unsigned long long diff) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (nb + KD_WARPS - 1) / KD_WARPS;
  const int w0 = w * per, w1 = min(nb, w0 + per);
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = pass * 8;
    if (((diff >> shift) & 0xFFull) == 0) continue;
    for (int i = tid; i < KD_HIST; i += KD_THREADS) hist[i] = 0;
    __syncthreads();
    for (int e0 = w0; e0 < w1; e0 += 32) {
      const int e = e0 + lane;
      const bool valid = e < w1;
      const uint32_t d = valid ? (uint32_t)((A[e] >> shift) & 0xFF) : 0u;
      const uint32_t peers = warp_digit_peers(d, valid);
      if (valid && (peers & lanemask_lt_kd()) == 0) hist[hidx(d, w)] += __popc(peers);
    }
    __syncthreads();
    block_exscan_4096(hist, wtot);
    for (int e0 = w0; e0 < w1; e0 += 32) {
      const int e = e0 + lane;
      const bool valid = e < w1;
      const unsigned long long k = valid ? A[e] : 0ull;
      const uint32_t d = valid ? (uint32_t)((k >> shift) & 0xFF) : 0u;
      const uint32_t peers = warp_digit_peers(d, valid);
      if (valid) B[hist[hidx(d, w)] + __popc(peers & lanemask_lt_kd())] = k;
      __syncwarp();
      if (valid && (peers & lanemask_lt_kd()) == 0) hist[hidx(d, w)] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    unsigned long long *t = A;
    A = B;
    B = t;
  }
  return A;
}

// Register-resident variant for bins of up to KD_REG_MAX points, sorted in
// place in one shared-memory array: per pass each warp reads its segment's
// keys once into registers, counts digits and records, per key, its rank
// among the warp's earlier keys of the same digit; after the block scan the
// keys go straight to their places (no second read, no read-modify-write).
constexpr int KD_ITEMS = 24;                                // keys per lane
constexpr int KD_REG_MAX = KD_ITEMS * 32 * KD_WARPS;        // 12288

__device__ void cta_radix_sort_reg(unsigned long long *A, int nb, uint32_t *hist, uint32_t *wtot,
                                   unsigned long long diff, int first_pass) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (nb + KD_WARPS - 1) / KD_WARPS;
  const int w0 = w * per, w1 = min(nb, w0 + per);
  const uint32_t lt = lanemask_lt_kd();
  for (int pass = first_pass; pass < 8; ++pass) {
    const int shift = pass * 8;
    if (((diff >> shift) & 0xFFull) == 0) continue;
    for (int i = tid; i < KD_HIST; i += KD_THREADS) hist[i] = 0;
    unsigned long long key[KD_ITEMS];
    // Per key: digit | rank among the item's earlier lanes of the digit << 8
    // | the digit group's lowest lane << 13 | (group size, on that lane) << 18.
    // The items are independent here (no shared-memory writes), so their
    // loads and ballots overlap.
    uint32_t code[KD_ITEMS];
#pragma unroll
    for (int i = 0; i < KD_ITEMS; ++i) {
      if (w0 + 32 * i < w1) {  // warp-uniform
        const int e = w0 + 32 * i + lane;
        const bool valid = e < w1;
        key[i] = valid ? A[e] : 0ull;
        const uint32_t d = valid ? (uint32_t)((key[i] >> shift) & 0xFFull) : 0u;
        const uint32_t peers = warp_digit_peers(d, valid);
        const uint32_t below = peers & lt;
        const uint32_t cnt = (valid && below == 0) ? (uint32_t)__popc(peers) : 0u;
        code[i] = d | ((uint32_t)__popc(below) << 8) | ((uint32_t)(__ffs(peers) - 1) << 13) | (cnt << 18);
      }
    }
    __syncthreads();  // counters zeroed
    // Running per-(digit, warp) counts, item by item: the only serial chain
    // is the group leaders' read-add-write of their counters.
#pragma unroll
    for (int i = 0; i < KD_ITEMS; ++i) {
      if (w0 + 32 * i < w1) {
        const uint32_t cd = code[i], d = cd & 0xFFu, cnt = cd >> 18;
        uint32_t old = 0;
        if (cnt) {
          old = hist[hidx(d, w)];
          hist[hidx(d, w)] = old + cnt;
        }
        old = __shfl_sync(0xffffffffu, old, (int)((cd >> 13) & 31u));
        code[i] = d | ((old + ((cd >> 8) & 31u)) << 8);
        __syncwarp();
      }
    }
    __syncthreads();
    block_exscan_4096(hist, wtot);
#pragma unroll
    for (int i = 0; i < KD_ITEMS; ++i) {
      const int e = w0 + 32 * i + lane;
      if (w0 + 32 * i < w1 && e < w1) A[hist[hidx(code[i] & 0xFFu, w)] + (code[i] >> 8)] = key[i];
    }
    __syncthreads();
  }
}

// The bin sum in 128-bit unsigned fixed point (lo, hi), exactly: a value
// m 2^(e - 1075) (m < 2^53, e the biased exponent, 1 for subnormals) is
// added as m 2^(e - emax + fxb), where emax is the largest value's exponent
// and fxb = 74 - ceil(log2 N_b), so N_b terms stay below 2^127.  Terms of a
// negative exponent are truncated (each below 2^-(fxb + 52) of the largest
// value).  Integer operations only.
__device__ __forceinline__ void fx_add(unsigned long long &lo, unsigned long long &hi, unsigned long long kb,
                                       int emax, int fxb) {
  const int e = (int)(kb >> 52);
  const unsigned long long m = (kb & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int sh = max(e, 1) - emax + fxb;
  unsigned long long tl = 0, th = 0;
  if (sh >= 64) {
    th = m << (sh - 64);
  } else if (sh > 0) {
    tl = m << sh;
    th = m >> (64 - sh);
  } else if (sh > -53) {
    tl = m >> -sh;
  }
  lo += tl;
  hi += th + (lo < tl);
}

// Bucket sort of a bin held in shared memory: the keys' range [kmin, kmax]
// is cut into KD_NBUCKET buckets of equal width in key space (the key bits
// are monotone in the value and close to its logarithm), the keys are
// counted and scattered into B by bucket (shared-memory atomics, any order
// within a bucket), and each key's place is its bucket's start plus the
// number of keys of the bucket that are smaller, or equal and earlier in B.
// Equal keys are equal values, so the result does not depend on the scatter
// order.  The ranking is quadratic in the bucket size: when a bucket holds
// more than KD_BUCKET_MAX keys this returns false with A untouched, and the
// caller radix-sorts instead.
constexpr int KD_NBUCKET = KD_THREADS * 8;  // block_exscan_4096's counters
static_assert(KD_NBUCKET == 4096, "the bucket passes use block_exscan_4096");
static_assert((KD_THREADS & (KD_THREADS - 1)) == 0, "the key order of the bucket passes needs a power of 2");
constexpr int KD_BUCKET_MAX = 512;

__device__ __forceinline__ int hpad(int b) { return b + (b >> 4); }  // block_exscan_4096's layout

// What the last step of a bucket sort can do with each key at its place
// besides storing it: with LOGS, it stores L = ln max(k, floor) (as the
// float-float pair log_ff gives) in place of the key, writes the key to the
// sorted output, if any, and adds it to the thread's 128-bit bin sum, so
// that no separate pass over the sorted keys is needed.
struct KeyLogs {
  const float2 *lnc, *invc;
  unsigned long long floor_bits;
  double *kg;  // sorted output of the bin, or NULL
  int emax, fxb;
};

template <bool LOGS>
__device__ bool cta_bucket_sort(unsigned long long *A, unsigned long long *B, int nb, uint32_t *hist,
                                uint32_t *wtot, unsigned long long kmin, unsigned long long kmax,
                                const KeyLogs &kl, unsigned long long &fx_lo, unsigned long long &fx_hi) {
  const int tid = threadIdx.x;
  const int sh = max(0, 64 - __clzll((long long)(kmax - kmin)) - 12);  // (kmax - kmin) >> sh < 4096
  for (int i = tid; i < KD_HIST; i += KD_THREADS) hist[i] = 0;
  __syncthreads();
  // neighbouring grid points have close values: the lanes of a warp take keys
  // 97 apart, so that their atomics mostly go to different counters
  const int pt = (tid * 97) & (KD_THREADS - 1);
  for (int j0 = 0; j0 < nb; j0 += KD_THREADS) {
    const int j = j0 + pt;
    if (j < nb) atomicAdd(&hist[hpad((int)((A[j] - kmin) >> sh))], 1u);
  }
  __syncthreads();
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) m = max(m, hist[hpad(tid * 8 + i)]);
  if (__syncthreads_or(m > (uint32_t)KD_BUCKET_MAX)) return false;
  block_exscan_4096(hist, wtot);  // bucket starts
  for (int j0 = 0; j0 < nb; j0 += KD_THREADS) {
    const int j = j0 + pt;
    if (j < nb) {
      const unsigned long long k = A[j];
      B[atomicAdd(&hist[hpad((int)((k - kmin) >> sh))], 1u)] = k;
    }
  }
  __syncthreads();  // hist now holds each bucket's end
  for (int j = tid; j < nb; j += KD_THREADS) {
    const unsigned long long k = B[j];
    const int b = (int)((k - kmin) >> sh);
    const int lo = b > 0 ? (int)hist[hpad(b - 1)] : 0, hi = (int)hist[hpad(b)];
    int r = lo;
    for (int i = lo; i < hi; ++i) {
      const unsigned long long x = B[i];
      r += (x < k) || (x == k && i < j);
    }
    if (LOGS) {
      if (kl.kg) kl.kg[r] = __longlong_as_double((long long)k);
      fx_add(fx_lo, fx_hi, k, kl.emax, kl.fxb);
      // non-negative doubles order as their bit patterns: max(k, floor) on the bits
      reinterpret_cast<float2 *>(A)[r] = log_ff(k > kl.floor_bits ? k : kl.floor_bits, kl.lnc, kl.invc);
    } else {
      A[r] = k;
    }
  }
  __syncthreads();
  return true;
}

// Sort by the high 32 bits (sign, exponent, top 20 fraction bits) first: 4
// passes instead of 8.  Keys that share their high word then sit together in
// their input order; runs of such ties are put in order by one thread each
// (insertion sort, runs of up to KD_RUN_MAX keys).  Ties are rare and short
// (relative differences below 2^-20); runs that are long and out of order
// make the CTA sort the reloaded keys by all 8 bytes instead.  Returns
// through `A` the keys in ascending order.
constexpr int KD_RUN_MAX = 64;

__device__ void cta_sort_bin(unsigned long long *A, const double *__restrict__ src, int nb, uint32_t *hist,
                             uint32_t *wtot, unsigned long long diff) {
  const int tid = threadIdx.x;
  cta_radix_sort_reg(A, nb, hist, wtot, diff, 4);
  // adjacent keys with equal high words in the wrong order?
  bool bad = false;
  for (int j = tid + 1; j < nb; j += KD_THREADS) {
    const unsigned long long a = A[j - 1], b = A[j];
    bad |= (a >> 32) == (b >> 32) && b < a;
  }
  if (!__syncthreads_or(bad)) return;
  bool too_long = false;
  for (int j = tid; j < nb; j += KD_THREADS) {
    const uint32_t h = (uint32_t)(A[j] >> 32);
    const bool start = (j == 0 || (uint32_t)(A[j - 1] >> 32) != h) && j + 1 < nb &&
                       (uint32_t)(A[j + 1] >> 32) == h;
    if (!start) continue;
    int e = j + 1;
    while (e < nb && e - j <= KD_RUN_MAX && (uint32_t)(A[e] >> 32) == h) ++e;
    if (e - j > KD_RUN_MAX) {
      too_long = true;
      continue;
    }
    for (int q = j + 1; q < e; ++q) {  // insertion sort of the run
      const unsigned long long v = A[q];
      int r = q - 1;
      while (r >= j && A[r] > v) {
        A[r + 1] = A[r];
        --r;
      }
      A[r + 1] = v;
    }
  }
  if (!__syncthreads_or(too_long)) return;
  for (int j = tid; j < nb; j += KD_THREADS) A[j] = (unsigned long long)__double_as_longlong(src[j]);
  __syncthreads();
  cta_radix_sort_reg(A, nb, hist, wtot, diff, 0);
}

// a + b for float-float pairs (two-sum of the high parts, low parts added)
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  float e = (a.x - (s - bb)) + (b.x - bb);
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// L_j + L_{nb-1-j} and L_j - L_{nb-1-j} (the middle point of an odd bin:
// L_j alone) as float-float pairs
__device__ __forceinline__ void fold_pair(const float2 *Ls, int nb, int j, float2 &Lp, float2 &Lm) {
  const float2 La = Ls[j];
  const int jm = nb - 1 - j;
  Lp = La;
  Lm = La;
  if (jm != j) {
    const float2 Lb = Ls[jm];
    Lp = ff_add(La, Lb);
    Lm = ff_add(La, make_float2(-Lb.x, -Lb.y));
  }
}

// c_k += P_kj L_j in double-float: (sh, sl) holds the running sum; the
// product of the high parts is exact as p + e (two-product), p joins sh by
// two-sum, and e, the two-sum error and the cross terms go to sl.
__device__ __forceinline__ void dfma_acc(float &sh, float &sl, float2 P, float2 L) {
  const float p = P.x * L.x;
  const float e = fmaf(P.x, L.x, -p);
  const float t = sh + p;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl += err + (e + fmaf(P.x, L.y, P.y * L.x));
}

__device__ __forceinline__ void fx_warp_sum(unsigned long long &lo, unsigned long long &hi) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o);
    const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, o);
    lo += l2;
    hi += h2 + (lo < l2);
  }
}

__device__ __forceinline__ float2 shfl_xor_f2(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Warp sums of eight float-float values by reduce-scatter: each exchange
// halves the values a lane carries, so lane l ends with the warp's sum of
// value l >> 2 (18 shuffle pairs instead of 40 for eight plain reductions).
__device__ __forceinline__ float2 ff_warp_sum8(const float2 (&v)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float2 v4[4], v2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 keep = b4 ? v[i + 4] : v[i], send = b4 ? v[i] : v[i + 4];
    v4[i] = ff_add(keep, shfl_xor_f2(send, 16));
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float2 keep = b3 ? v4[i + 2] : v4[i], send = b3 ? v4[i] : v4[i + 2];
    v2[i] = ff_add(keep, shfl_xor_f2(send, 8));
  }
  float2 r = ff_add(b2 ? v2[1] : v2[0], shfl_xor_f2(b2 ? v2[0] : v2[1], 4));
  r = ff_add(r, shfl_xor_f2(r, 2));
  return ff_add(r, shfl_xor_f2(r, 1));
}

// Per-bin sort + fit.  MODE 0: keys in shared memory (nb <= KD_REG_MAX, two
// arrays: bucket sort, else register-resident radix passes); MODE 1: keys in
// the global ping-pong
// buffers gA, gB.  P holds the pseudo-inverse as split pairs [k][j].
// FIT = false: the bin's fit is left to k_kdist_fit; the kernel writes the
// folded logarithms (L_j + L_{nb-1-j}, L_j - L_{nb-1-j}) for j < nh, as
// float-float pairs, to Lf[bin * npad + j] (npad = nh rounded up to 32,
// zero past nh), and no coefficients.
// FIT = true: it fits the bin itself from P in global memory (the
// allocation-free entry point, which has no room for Lf).  The two are
// separate instantiations so that each carries only its own code.  Bins
// that fit in shared memory once take k_kdist_rank instead of MODE 0 with
// FIT = false.
template <int MODE, bool FIT>
__global__ void __launch_bounds__(KD_THREADS)
    k_kdist_bin(const double *__restrict__ kappa, int nb, int ncheb, double kappa_floor,
                const float2 *__restrict__ P, const float2 *__restrict__ lntab, unsigned long long *gA,
                unsigned long long *gB, double *__restrict__ coef, double *__restrict__ mean,
                double *__restrict__ kg_out, float4 *__restrict__ Lf) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t hist[KD_HIST];
  __shared__ uint32_t wtot[32];
  __shared__ unsigned long long red_and[KD_WARPS], red_or[KD_WARPS], red_min[KD_WARPS], red_max[KD_WARPS];
  __shared__ float2 red[KD_WARPS][NCHEB_MAX];
  __shared__ unsigned long long red_fx[KD_WARPS][2];
  __shared__ float2 s_lnc[128], s_invc[128];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t off = (int64_t)blockIdx.x * nb;
  unsigned long long *A = MODE == 0 ? (unsigned long long *)dsm : gA + off;
  unsigned long long vand = ~0ull, vor = 0ull, vmin = ~0ull, vmax = 0ull;
  for (int j = tid; j < nb; j += KD_THREADS) {
    const unsigned long long k = (unsigned long long)__double_as_longlong(kappa[off + j]);
    A[j] = k;
    vand &= k;
    vor |= k;
    vmin = min(vmin, k);
    vmax = max(vmax, k);
  }
  if (tid < KD_LNTAB) {  // ln c_j and 1/c_j as FP32 (high, low) pairs
    const float2 t = lntab[tid];
    if (tid < 128)
      s_lnc[tid] = t;
    else
      s_invc[tid - 128] = t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    vand &= __shfl_down_sync(0xffffffffu, vand, o);
    vor |= __shfl_down_sync(0xffffffffu, vor, o);
    vmin = min(vmin, __shfl_down_sync(0xffffffffu, vmin, o));
    vmax = max(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
  }
  if (lane == 0) {
    red_and[w] = vand;
    red_or[w] = vor;
    red_min[w] = vmin;
    red_max[w] = vmax;
  }
  __syncthreads();
  vand = ~0ull;
  vor = 0ull;
  vmin = ~0ull;
  vmax = 0ull;
  for (int i = 0; i < KD_WARPS; ++i) {
    vand &= red_and[i];
    vor |= red_or[i];
    vmin = min(vmin, red_min[i]);
    vmax = max(vmax, red_max[i]);
  }
  // the bin sum (128-bit fixed point, relative to the largest key) and the
  // logarithms' arguments
  const unsigned long long kmax = vmax;
  const int emax = max((int)(kmax >> 52), 1);
  const int fxb = 74 - (nb > 1 ? 32 - __clz(nb - 1) : 0);
  unsigned long long fx_lo = 0, fx_hi = 0;
  const unsigned long long floor_bits = (unsigned long long)__double_as_longlong(kappa_floor);
  const KeyLogs kl{s_lnc, s_invc, floor_bits, kg_out ? kg_out + off : nullptr, emax, fxb};
  bool logged = false;  // the bucket sort's last step took the logarithms
  unsigned long long *S;
  if (MODE == 0) {
    // the second key array of the bucket sort follows A in shared memory
    if (vmin != vmax) {
      logged = cta_bucket_sort<true>(A, A + nb, nb, hist, wtot, vmin, vmax, kl, fx_lo, fx_hi);
      if (!logged) cta_sort_bin(A, kappa + off, nb, hist, wtot, vand ^ vor);
    }
    S = A;
  } else {
    // bins too large for shared memory: the same bucket sort through the
    // global ping-pong buffers (about 11 accesses a key against 24 for the
    // eight radix passes), the radix passes when a bucket is too full
    if (vmin == vmax || cta_bucket_sort<false>(A, gB + off, nb, hist, wtot, vmin, vmax, kl, fx_lo, fx_hi))
      S = A;
    else
      S = cta_radix_sort(A, gB + off, nb, hist, wtot, vand ^ vor);
  }
  // sorted values out, the bin sum, and L_j in place as a split pair
  float2 *Ls = reinterpret_cast<float2 *>(S);
  __syncthreads();
  // four points a thread per pass: their keys are read before any L_j is
  // written in place, so the four logarithms run side by side (the integer
  // bin sum does not depend on the order)
  constexpr int LU = 4;
  for (int j0 = logged ? nb : tid; j0 < nb; j0 += LU * KD_THREADS) {
    unsigned long long kq[LU];
#pragma unroll
    for (int q = 0; q < LU; ++q) {
      const int j = j0 + q * KD_THREADS;
      kq[q] = j < nb ? S[j] : 0ull;
    }
    float2 lq[LU];
#pragma unroll
    for (int q = 0; q < LU; ++q) {
      const int j = j0 + q * KD_THREADS;
      if (j < nb) {
        if (kg_out) kg_out[off + j] = __longlong_as_double((long long)kq[q]);
        fx_add(fx_lo, fx_hi, kq[q], emax, fxb);
      }
      // non-negative doubles order as their bit patterns: max(k, floor) on the bits
      lq[q] = log_ff(kq[q] > floor_bits ? kq[q] : floor_bits, s_lnc, s_invc);
    }
#pragma unroll
    for (int q = 0; q < LU; ++q) {
      const int j = j0 + q * KD_THREADS;
      if (j < nb) Ls[j] = lq[q];
    }
  }
  fx_warp_sum(fx_lo, fx_hi);
  if (lane == 0) {
    red_fx[w][0] = fx_lo;
    red_fx[w][1] = fx_hi;
  }
  __syncthreads();
  const int nh = (nb + 1) >> 1;
  if (!FIT) {
    // folded logarithms for k_kdist_fit (the middle point of an odd bin
    // once, in both halves of its pair)
    const int npad = ((nh + 31) >> 5) << 5;
    float4 *out = Lf + (int64_t)blockIdx.x * npad;
    for (int jj = tid; jj < npad; jj += KD_THREADS) {
      float2 Lp = make_float2(0.0f, 0.0f), Lm = Lp;
      if (jj < nh) fold_pair(Ls, nb, jj, Lp, Lm);
      out[jj] = make_float4(Lp.x, Lp.y, Lm.x, Lm.y);
    }
  } else {
    // c = P L, eight coefficients per sweep over the first half of the
    // points: c_k = sum_{j < nh} P[k][j] (L_j + (-1)^k L_{nb-1-j}) (the
    // middle point of an odd bin once), P the blocked symmetrized half
    for (int k0 = 0; k0 < ncheb; k0 += 8) {
      float sh[8], sl[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q] = sl[q] = 0.0f;
      // two points a step, so that 16 loads of P are in flight per thread
      for (int jj = tid; jj < nh; jj += 2 * KD_THREADS) {
        const int j2 = jj + KD_THREADS;
        float2 Pa[8], Pb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          Pa[q] = k0 + q < ncheb ? P[pinv_index(k0 + q, jj, ncheb)] : make_float2(0.0f, 0.0f);
          Pb[q] = (k0 + q < ncheb && j2 < nh) ? P[pinv_index(k0 + q, j2, ncheb)] : make_float2(0.0f, 0.0f);
        }
        float2 Lp, Lm;
        fold_pair(Ls, nb, jj, Lp, Lm);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (k0 + q < ncheb) dfma_acc(sh[q], sl[q], Pa[q], (q & 1) ? Lm : Lp);
        if (j2 < nh) {
          fold_pair(Ls, nb, j2, Lp, Lm);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (k0 + q < ncheb) dfma_acc(sh[q], sl[q], Pb[q], (q & 1) ? Lm : Lp);
        }
      }
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float h, l;
        two_sum_f(sh[q], sl[q], h, l);
        v[q] = make_float2(h, l);
      }
      const float2 r = ff_warp_sum8(v, lane);
      if ((lane & 3) == 0 && k0 + (lane >> 2) < ncheb) red[w][k0 + (lane >> 2)] = r;
    }
  }
  __syncthreads();
  if (FIT && tid < ncheb) {
    float2 s = red[0][tid];
    for (int i = 1; i < KD_WARPS; ++i) s = ff_add(s, red[i][tid]);
    coef[(int64_t)blockIdx.x * ncheb + tid] = (double)s.x + (double)s.y;
  }
  if (tid == NCHEB_MAX && mean) {
    unsigned long long lo = 0, hi = 0;
    for (int i = 0; i < KD_WARPS; ++i) {
      lo += red_fx[i][0];
      hi += red_fx[i][1] + (lo < red_fx[i][0]);
    }
    double m;
    if ((kmax >> 52) >= 0x7FF)  // infinite or NaN largest value (or a negative one)
      m = (kmax >> 63) ? __longlong_as_double(0x7FF8000000000000ll) : __longlong_as_double((long long)kmax);
    else
      m = ldexp(fma((double)hi, 0x1p64, (double)lo), emax - 1075 - fxb) / (double)nb;
    mean[blockIdx.x] = m;
  }
}

// ---------------------------------------------- bins in shared memory --
// The per-bin stage (FIT = false) for bins whose keys fit in shared memory
// once: 8 B a point for the key, 2 B for its place.  The keys are read from
// kappa three times (the range from HBM, then the bucket counts and the
// scatter from L2), so that shared memory holds only the keys in bucket
// order, the bucket counters are 16-bit, and two CTAs of a 10^4-point bin
// share an SM (the barrier-separated phases of one overlap the other's).
// Each key's rank is its bucket's start plus the keys of the bucket that
// are smaller, or equal and earlier (as in cta_bucket_sort); the rank pass
// records, per sorted place, the key's position in B, and a last pass takes
// the places in order, each with its mirror nb-1-j, and writes their outputs
// with coalesced stores (pair_out): the sorted values, their terms of the
// bin sum, and the folded logarithms of L = ln max(k, floor).  A bucket of more than KD_BUCKET_MAX
// keys is ranked by position when all its keys are equal (a run of zeros or
// of one floor value: equal keys are equal values); any other such bucket
// sends the bin to the radix passes through the global buffers gA, gB.
struct BinOut {
  const float2 *lnc, *invc;
  unsigned long long floor_bits;
  double *kg;  // the bin's sorted output, or NULL
  float4 *X;   // the bin's row of folded logarithms
  int nb, emax, fxb;
};

// The outputs of sorted place j < nh and of its mirror nb-1-j, from their
// keys ka and kb: the sorted values, their terms of the bin sum, and the
// folded logarithms (L_j + L_{nb-1-j}, L_j - L_{nb-1-j}) as float-float
// pairs in X[j] (the middle point of an odd bin: L_j in both).  The two
// logarithms run side by side.
__device__ __forceinline__ void pair_out(const BinOut &o, int j, unsigned long long ka, unsigned long long kb,
                                         unsigned long long &fx_lo, unsigned long long &fx_hi) {
  const int m = o.nb - 1 - j;
  // non-negative doubles order as their bit patterns: max(k, floor) on the bits
  const float2 La = log_ff(ka > o.floor_bits ? ka : o.floor_bits, o.lnc, o.invc);
  const float2 Lb = log_ff(kb > o.floor_bits ? kb : o.floor_bits, o.lnc, o.invc);
  if (o.kg) o.kg[j] = __longlong_as_double((long long)ka);
  fx_add(fx_lo, fx_hi, ka, o.emax, o.fxb);
  float2 Lp = La, Lm = La;
  if (m != j) {
    if (o.kg) o.kg[m] = __longlong_as_double((long long)kb);
    fx_add(fx_lo, fx_hi, kb, o.emax, o.fxb);
    Lp = ff_add(La, Lb);
    Lm = ff_add(La, make_float2(-Lb.x, -Lb.y));
  }
  o.X[j] = make_float4(Lp.x, Lp.y, Lm.x, Lm.y);
}

// The bucket counters of k_kdist_rank as 16-bit halves of 32-bit words
// (bins of fewer than 2^16 points): bucket b in half b & 1 of word b >> 1,
// the words padded by one every 16 (fewer bank conflicts in the scan).
constexpr int KR_HWORDS = KD_NBUCKET / 2 + KD_NBUCKET / 32;
__device__ __forceinline__ int hw_idx(int wi) { return wi + (wi >> 4); }
__device__ __forceinline__ uint32_t hw_get(const uint32_t *hw, int b) {
  return (hw[hw_idx(b >> 1)] >> ((b & 1) << 4)) & 0xFFFFu;
}
// returns the bucket's counter before the increment
__device__ __forceinline__ uint32_t hw_inc(uint32_t *hw, int b) {
  const int s = (b & 1) << 4;
  return (atomicAdd(&hw[hw_idx(b >> 1)], 1u << s) >> s) & 0xFFFFu;
}

// Exclusive scan of the KD_NBUCKET packed counters in bucket order, in place
// (every partial sum below 2^16).
__device__ void block_exscan_4096_u16(uint32_t *hw, uint32_t *wtot) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t loc[4];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    loc[i] = hw[hw_idx(tid * 4 + i)];
    s += (loc[i] & 0xFFFFu) + (loc[i] >> 16);
  }
  uint32_t v = s;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wtot[w] = v;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < KD_WARPS ? wtot[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane < KD_WARPS) wtot[lane] = x;
  }
  __syncthreads();
  uint32_t run = v - s + (w > 0 ? wtot[w - 1] : 0u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = run;
    run += loc[i] & 0xFFFFu;
    hw[hw_idx(tid * 4 + i)] = lo | (run << 16);
    run += loc[i] >> 16;
  }
  __syncthreads();
}

// A key's place in the bin from its bucket in B (bucket ends in hw): the
// bucket's start plus its keys that are smaller, or equal and earlier in B;
// a bucket of more than KD_BUCKET_MAX keys holds one value (checked by the
// caller), so its keys take their places in B.
__device__ __forceinline__ int bucket_rank(const unsigned long long *B, const uint32_t *hw, unsigned long long k,
                                           int p, unsigned long long vmin, int sh) {
  const int b = (int)((k - vmin) >> sh);
  const int lo = b > 0 ? (int)hw_get(hw, b - 1) : 0, hi = (int)hw_get(hw, b);
  if (hi - lo > KD_BUCKET_MAX) return p;
  int r = lo;
  for (int i = lo; i < hi; ++i) {
    const unsigned long long x = B[i];
    r += (x < k) || (x == k && i < p);
  }
  return r;
}

constexpr int KR_UNROLL = 4;  // keys a thread has in flight in the passes over kappa

__global__ void __launch_bounds__(KD_THREADS, 2)
    k_kdist_rank(const double *__restrict__ kappa, int nb, int npad, double kappa_floor,
                 const float2 *__restrict__ lntab, unsigned long long *gA, unsigned long long *gB,
                 double *__restrict__ mean, double *__restrict__ kg_out, float4 *__restrict__ X) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t hw[KR_HWORDS];
  __shared__ uint32_t wtot[32];
  __shared__ unsigned long long red[4][KD_WARPS];
  __shared__ unsigned long long red_fx[KD_WARPS][2];
  __shared__ float2 s_lnc[128], s_invc[128];
  // keys in bucket order, then each sorted place's position in B (16 bits)
  unsigned long long *B = reinterpret_cast<unsigned long long *>(dsm);
  uint16_t *Q = reinterpret_cast<uint16_t *>(dsm + (size_t)nb * 8);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t off = (int64_t)blockIdx.x * nb;
  const unsigned long long *K = reinterpret_cast<const unsigned long long *>(kappa + off);
  // the keys' range (and the bits in which they differ, for the radix passes)
  unsigned long long vand = ~0ull, vor = 0ull, vmin = ~0ull, vmax = 0ull;
  for (int j0 = tid; j0 < nb; j0 += KR_UNROLL * KD_THREADS) {
    unsigned long long kq[KR_UNROLL];
#pragma unroll
    for (int q = 0; q < KR_UNROLL; ++q) {
      const int j = j0 + q * KD_THREADS;
      kq[q] = K[j < nb ? j : j0];  // a repeat of a key changes none of the four
    }
#pragma unroll
    for (int q = 0; q < KR_UNROLL; ++q) {
      vand &= kq[q];
      vor |= kq[q];
      vmin = min(vmin, kq[q]);
      vmax = max(vmax, kq[q]);
    }
  }
  if (tid < KD_LNTAB) {  // ln c_j and 1/c_j as FP32 (high, low) pairs
    const float2 t = lntab[tid];
    if (tid < 128)
      s_lnc[tid] = t;
    else
      s_invc[tid - 128] = t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    vand &= __shfl_down_sync(0xffffffffu, vand, o);
    vor |= __shfl_down_sync(0xffffffffu, vor, o);
    vmin = min(vmin, __shfl_down_sync(0xffffffffu, vmin, o));
    vmax = max(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
  }
  if (lane == 0) {
    red[0][w] = vand;
    red[1][w] = vor;
    red[2][w] = vmin;
    red[3][w] = vmax;
  }
  const int nh = (nb + 1) >> 1;
  float4 *Xb = X + (int64_t)blockIdx.x * npad;
  for (int jj = nh + tid; jj < npad; jj += KD_THREADS) Xb[jj] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  __syncthreads();
  // (the bits of the AND, the OR and the largest key stay in `red` for the
  // radix passes and the mean)
  vmin = ~0ull;
  vmax = 0ull;
  for (int i = 0; i < KD_WARPS; ++i) {
    vmin = min(vmin, red[2][i]);
    vmax = max(vmax, red[3][i]);
  }
  const int emax = max((int)(vmax >> 52), 1);
  const int fxb = 74 - (nb > 1 ? 32 - __clz(nb - 1) : 0);
  const BinOut o{s_lnc, s_invc, (unsigned long long)__double_as_longlong(kappa_floor),
                 kg_out ? kg_out + off : nullptr, Xb, nb, emax, fxb};
  unsigned long long fx_lo = 0, fx_hi = 0;
  bool bucketed = true;  // CTA-uniform: false sends the bin to the radix passes
  if (vmin == vmax) {
    for (int j = tid; j < nh; j += KD_THREADS) pair_out(o, j, vmin, vmin, fx_lo, fx_hi);
  } else {
    const int sh = max(0, 64 - __clzll((long long)(vmax - vmin)) - 12);  // (vmax - vmin) >> sh < 4096
    for (int i = tid; i < KR_HWORDS; i += KD_THREADS) hw[i] = 0;
    __syncthreads();
    // neighbouring grid points have close values: the lanes of a warp take
    // keys 97 apart, so that their atomics mostly go to different counters
    const int pt = (tid * 97) & (KD_THREADS - 1);
    for (int j0 = pt; j0 < nb; j0 += KR_UNROLL * KD_THREADS) {
      unsigned long long kq[KR_UNROLL];
#pragma unroll
      for (int q = 0; q < KR_UNROLL; ++q) {
        const int j = j0 + q * KD_THREADS;
        kq[q] = j < nb ? K[j] : 0ull;
      }
#pragma unroll
      for (int q = 0; q < KR_UNROLL; ++q)
        if (j0 + q * KD_THREADS < nb) hw_inc(hw, (int)((kq[q] - vmin) >> sh));
    }
    __syncthreads();
    uint32_t mx = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) mx = max(mx, hw_get(hw, tid * 8 + i));
    const bool big = __syncthreads_or(mx > (uint32_t)KD_BUCKET_MAX);
    block_exscan_4096_u16(hw, wtot);  // bucket starts
    for (int j0 = pt; j0 < nb; j0 += KR_UNROLL * KD_THREADS) {
      unsigned long long kq[KR_UNROLL];
#pragma unroll
      for (int q = 0; q < KR_UNROLL; ++q) {
        const int j = j0 + q * KD_THREADS;
        kq[q] = j < nb ? K[j] : 0ull;
      }
#pragma unroll
      for (int q = 0; q < KR_UNROLL; ++q)
        if (j0 + q * KD_THREADS < nb) B[hw_inc(hw, (int)((kq[q] - vmin) >> sh))] = kq[q];
    }
    __syncthreads();  // hw now holds each bucket's end
    if (big) {
      // is every bucket over KD_BUCKET_MAX keys a run of one value?
      bool mixed = false;
      for (int p = tid; p < nb; p += KD_THREADS) {
        const unsigned long long k = B[p];
        const int b = (int)((k - vmin) >> sh);
        const int lo = b > 0 ? (int)hw_get(hw, b - 1) : 0, hi = (int)hw_get(hw, b);
        mixed |= hi - lo > KD_BUCKET_MAX && k != B[lo];
      }
      bucketed = !__syncthreads_or(mixed);
    }
    if (bucketed) {
      for (int p = tid; p < nb; p += KD_THREADS) Q[bucket_rank(B, hw, B[p], p, vmin, sh)] = (uint16_t)p;
      __syncthreads();
      for (int j = tid; j < nh; j += KD_THREADS) pair_out(o, j, B[Q[j]], B[Q[nb - 1 - j]], fx_lo, fx_hi);
    }
  }
  if (!bucketed) {
    unsigned long long *A = gA + off;
    for (int j = tid; j < nb; j += KD_THREADS) A[j] = K[j];
    vand = ~0ull;
    vor = 0ull;
    for (int i = 0; i < KD_WARPS; ++i) {
      vand &= red[0][i];
      vor |= red[1][i];
    }
    __syncthreads();
    // the radix passes' counters in the (now unused) key array
    const unsigned long long *S =
        cta_radix_sort(A, gB + off, nb, reinterpret_cast<uint32_t *>(dsm), wtot, vand ^ vor);
    for (int j = tid; j < nh; j += KD_THREADS) pair_out(o, j, S[j], S[nb - 1 - j], fx_lo, fx_hi);
  }
  fx_warp_sum(fx_lo, fx_hi);
  if (lane == 0) {
    red_fx[w][0] = fx_lo;
    red_fx[w][1] = fx_hi;
  }
  __syncthreads();
  if (tid == 0 && mean) {
    unsigned long long lo = 0, hi = 0, kmax = 0;
    for (int i = 0; i < KD_WARPS; ++i) {
      lo += red_fx[i][0];
      hi += red_fx[i][1] + (lo < red_fx[i][0]);
      kmax = max(kmax, red[3][i]);
    }
    double m;
    if ((kmax >> 52) >= 0x7FF)  // infinite or NaN largest value (or a negative one)
      m = (kmax >> 63) ? __longlong_as_double(0x7FF8000000000000ll) : __longlong_as_double((long long)kmax);
    else
      m = ldexp(fma((double)hi, 0x1p64, (double)lo), max((int)(kmax >> 52), 1) - 1075 - fxb) / (double)nb;
    mean[blockIdx.x] = m;
  }
}

// --------------------------------------------------------------- the fit --
// c = P L for many bins at once: a CTA takes KF_BINS bins (one warp each)
// and one group of P's column blocks, and streams them through shared
// memory in chunks of KF_COLS columns -- the chunk of P and, for each of its
// bins, the chunk of folded logarithms (L_j + L_{nb-1-j} for the even
// coefficients, L_j - L_{nb-1-j} for the odd ones) -- by cp.async,
// double-buffered so that the next chunk's copies fly while the current one
// is used.  So P is read from L2 once per KF_BINS bins instead of once per
// bin.  Every lane accumulates the ncheb coefficients of its bin over its
// columns in double-float (dfma_acc), the warp reduces them, and the partial sums of the column groups go to `part`
// ([group][bin][k]).  The last CTA of a row of bins to finish (counted in
// `done`, which it sets back to zero) adds the groups' partial sums in group
// order, so the result does not depend on which CTA finishes last.
constexpr int KF_BINS = 8;
constexpr int KF_THREADS = 32 * KF_BINS;
constexpr int KF_COLS = 128;  // columns (four 32-column blocks of P) per chunk

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Shared memory of k_kdist_fit: two stages of [P chunk | folded logs].
size_t kdist_fit_smem(int ncheb) {
  return 2 * ((size_t)ncheb * KF_COLS * sizeof(float2) + (size_t)KF_BINS * KF_COLS * sizeof(float4));
}

// NC: a compile-time bound on ncheb (8, 16, 20, 24 or 32), so that no
// issue slot goes to coefficients beyond it.
template <int NC>
__global__ void __launch_bounds__(KF_THREADS)
    k_kdist_fit(const float4 *__restrict__ Lf, int npad, int nbins, int ncheb, const float2 *__restrict__ P,
                int cols_per_group, float2 *__restrict__ part, unsigned int *__restrict__ done,
                double *__restrict__ coef) {
  extern __shared__ __align__(16) unsigned char kf_smem[];
  __shared__ float2 wred[KF_BINS][NCHEB_MAX];
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = blockIdx.x;
  const int bin = blockIdx.y * KF_BINS + w;
  const int c0 = g * cols_per_group, c1 = min(npad, c0 + cols_per_group);
  // stage st: [P chunk (ncheb x KF_COLS float2) | folded logs (KF_BINS x KF_COLS float4)]
  const size_t pbytes = (size_t)ncheb * KF_COLS * sizeof(float2);
  const size_t sbytes = pbytes + (size_t)KF_BINS * KF_COLS * sizeof(float4);
  auto Pst = [&](int st) { return reinterpret_cast<float2 *>(kf_smem + st * sbytes); };
  auto Lst = [&](int st) { return reinterpret_cast<float4 *>(kf_smem + st * sbytes + pbytes); };
  const int b0 = blockIdx.y * KF_BINS;
  // copies of the chunk at columns cc into stage st (each thread its share)
  auto issue = [&](int cc, int st) {
    const int ncol = min(KF_COLS, c1 - cc);  // a multiple of 32
    const float2 *src = P + (int64_t)(cc >> 5) * ncheb * 32;  // whole blocks, contiguous
    const int np = ncol * ncheb / 2;                          // 16-byte pieces of P
    for (int e = tid; e < np; e += KF_THREADS) cp_async16(Pst(st) + 2 * e, src + 2 * e);
    // the folded logs: warp wb copies its bin's row (ncol is a multiple of 32)
    {
      const int wb = tid >> 5;
      const float4 *row = Lf + (int64_t)min(b0 + wb, nbins - 1) * npad + cc;
      for (int cl = tid & 31; cl < ncol; cl += 32) cp_async16(Lst(st) + wb * KF_COLS + cl, row + cl);
    }
  };
  constexpr int NR = (NC + 7) / 8 * 8;  // accumulators, a multiple of the reduction's 8
  float sh[NR], sl[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) sh[k] = sl[k] = 0.0f;
  if (c0 < c1) issue(c0, 0);
  cp_async_commit();
  int st = 0;
  for (int cc = c0; cc < c1; cc += KF_COLS, st ^= 1) {
    if (cc + KF_COLS < c1) issue(cc + KF_COLS, st ^ 1);
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of the current chunk have landed
    __syncthreads();   // and everyone's
    const int ncol = min(KF_COLS, c1 - cc);
    if (bin < nbins) {
      if (ncheb == NC) {  // every accumulator used: no per-coefficient test
        for (int b = 0; b < (ncol >> 5); ++b) {
          const float4 l = Lst(st)[w * KF_COLS + 32 * b + lane];  // zero past nh
          const float2 Lp = make_float2(l.x, l.y), Lm = make_float2(l.z, l.w);
          const float2 *pb = Pst(st) + b * NC * 32 + lane;
#pragma unroll
          for (int k = 0; k < NC; ++k) dfma_acc(sh[k], sl[k], pb[k * 32], (k & 1) ? Lm : Lp);
        }
      } else {
        for (int b = 0; b < (ncol >> 5); ++b) {
          const float4 l = Lst(st)[w * KF_COLS + 32 * b + lane];  // zero past nh
          const float2 Lp = make_float2(l.x, l.y), Lm = make_float2(l.z, l.w);
          const float2 *pb = Pst(st) + b * ncheb * 32 + lane;
#pragma unroll
          for (int k = 0; k < NC; ++k)
            if (k < ncheb) dfma_acc(sh[k], sl[k], pb[k * 32], (k & 1) ? Lm : Lp);
        }
      }
    }
    __syncthreads();  // the stage is refilled two chunks on
  }
  // warp sums, eight coefficients at a time (reduce-scatter)
#pragma unroll
  for (int k0 = 0; k0 < NR; k0 += 8) {
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float h, l;
      two_sum_f(sh[k0 + q], sl[k0 + q], h, l);
      v[q] = make_float2(h, l);
    }
    const float2 r = ff_warp_sum8(v, lane);
    if ((lane & 3) == 0) wred[w][k0 + (lane >> 2)] = r;
  }
  __syncwarp();
  if (bin < nbins && lane < ncheb)
    part[((int64_t)g * nbins + bin) * ncheb + lane] = wred[w][lane];
  __threadfence();  // the partial sums are visible device-wide before the count
  __syncthreads();
  if (tid == 0) {
    const unsigned int prev = atomicAdd(&done[blockIdx.y], 1u);
    s_last = prev == gridDim.x - 1;
    if (s_last) done[blockIdx.y] = 0;  // every group has counted: ready for the next call
  }
  __syncthreads();
  if (s_last && bin < nbins && lane < ncheb) {
    __threadfence();
    const float2 *pe = part + (int64_t)bin * ncheb + lane;
    const int64_t gs = (int64_t)nbins * ncheb;
    float2 s = __ldcg(pe);
    for (int gg = 1; gg < (int)gridDim.x; ++gg) s = ff_add(s, __ldcg(pe + gg * gs));
    coef[(int64_t)bin * ncheb + lane] = (double)s.x + (double)s.y;
  }
}

int64_t kdist_fold_bytes(int64_t n, int nbins) {
  const int64_t nb = n / nbins, nh = (nb + 1) / 2, npad = (nh + 31) / 32 * 32;
  return (int64_t)nbins * npad * 16;
}

// Column groups of the fit: enough CTAs for two per SM, each group at least
// two chunks wide.
static int fit_groups(helk_ctx *c, int npad, int nbins) {
  const int bingroups = (nbins + KF_BINS - 1) / KF_BINS;
  const int want = std::max(1, (2 * c->num_sms + bingroups - 1) / bingroups);
  const int most = std::max(1, npad / (2 * KF_COLS));
  return std::min(want, most);
}

int64_t kdist_part_bytes(helk_ctx *c, int64_t n, int nbins) {
  const int64_t nb = n / nbins, nh = (nb + 1) / 2, npad = (nh + 31) / 32 * 32;
  return (int64_t)fit_groups(c, (int)npad, nbins) * nbins * NCHEB_MAX * 8;
}

int64_t kdist_done_bytes(int nbins) { return (int64_t)((nbins + KF_BINS - 1) / KF_BINS) * 4; }

int64_t kdist_smem_max_points(helk_ctx *c) {
  // k_kdist_rank: the keys (8 B a point) and their sorted places (2 B)
  // beside its static shared memory
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_kdist_rank) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int64_t avail = (int64_t)c->max_smem_optin - (int64_t)fa.sharedSizeBytes - 16;
  return std::min<int64_t>(65535, avail > 0 ? avail / 10 : 0);  // 16-bit counters and places
}

// k_kdist_rank's dynamic shared memory: the keys and their 16-bit places,
// at least the radix passes' counters (which reuse it).
static size_t kdist_rank_smem(int nb) {
  return std::max<size_t>(((size_t)nb * 10 + 15) / 16 * 16, (size_t)KD_HIST * 4);
}

cudaError_t launch_kdist_bins(helk_ctx *c, const double *kappa, int64_t n, int nbins, int ncheb,
                              double kappa_floor, double *coef, double *mean, double *kg_out) {
  const int nb = (int)(n / nbins);
  const float2 *P = reinterpret_cast<const float2 *>(c->pinv);
  const float2 *lntab = pinv_lntab(c, nb, ncheb);
  float4 *Lf = reinterpret_cast<float4 *>(c->kd_fold);
  const int nh = (nb + 1) / 2, npad = (nh + 31) / 32 * 32;
  if ((int64_t)nb <= kdist_smem_max_points(c)) {
    const size_t smem = kdist_rank_smem(nb);
    cudaError_t e = cudaFuncSetAttribute(k_kdist_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ++c->launches;
    k_kdist_rank<<<nbins, KD_THREADS, smem, c->stream>>>(kappa, nb, npad, kappa_floor, lntab, c->sort_a,
                                                         c->sort_b, mean, kg_out, Lf);
  } else {
    ++c->launches;
    k_kdist_bin<1, false><<<nbins, KD_THREADS, 0, c->stream>>>(kappa, nb, ncheb, kappa_floor, P, lntab,
                                                               c->sort_a, c->sort_b, coef, mean, kg_out, Lf);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int groups = fit_groups(c, npad, nbins);
  const int cpg = ((npad / 32 + groups - 1) / groups) * 32;
  float2 *part = reinterpret_cast<float2 *>(c->kd_part);
  const size_t fsm = kdist_fit_smem(ncheb);
  auto fit = ncheb <= 8 ? k_kdist_fit<8> : ncheb <= 16 ? k_kdist_fit<16> : ncheb <= 20 ? k_kdist_fit<20>
           : ncheb <= 24 ? k_kdist_fit<24> : k_kdist_fit<32>;
  e = cudaFuncSetAttribute(fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
  if (e != cudaSuccess) return e;
  ++c->launches;
  fit<<<dim3(groups, (nbins + KF_BINS - 1) / KF_BINS), KF_THREADS, fsm, c->stream>>>(
      Lf, npad, nbins, ncheb, P, cpg, part, reinterpret_cast<unsigned int *>(c->kd_done), coef);
  return cudaGetLastError();
}

// ---------------------------------------------------------- transmission --
// T_b(m) = int_0^1 exp(-k(g) m) dg per bin b and column mass m (Sec. 2.1):
// from the sorted values by the midpoint rule on g_j = (j + 1/2)/N_b, and
// from the Chebyshev fit by the midpoint rule on ng points.
//
// The smallest value k_0 of a bin is factored out: T = e^{-k_0 m} S / N,
// S = sum_j e^{-d_j}, d_j = (k_j - k_0) m >= 0, so S lies in [1, N] and each
// term in (0, 1].  Terms with d_j >= 87 are below 2^-125 of S and left out
// (for sorted values: every term from the first such j on, found by a binary
// search); the rest are evaluated on the FP32 pipe as float-float pairs:
// k_j - k_0 is formed once per point in FP64 and kept as a pair D_j scaled
// by the bin's 2^-F (F the exponent of the largest difference), d_j = D_j M
// with M = m 2^F, and e^{-d} by a table-driven exponential (Tang 1989):
// d = (n/256) ln 2 - r with |r| <= ln2/512, e^{-d} = 2^{-n/256} e^r,
// 2^{-j/256} from a 256-entry table of pairs and e^r = 1 + r + (r^2/2)(1 +
// r/3 + r^2/12), the bracket's small part in FP32 (relative error of a term
// ~5e-15, set by the table's pairs).  Differences below 2^(F-100),
// whose pairs would lose precision, take FP64 exp; equal values add 1 each.
// One FP64 exponential per (bin, m) for e^{-k_0 m}.  Bins whose values are
// not sorted, finite and non-negative take the plain FP64 sum.
constexpr int TR_THREADS = 256;
constexpr double TR_DMAX = 87.0;  // e^-87 < 2^-125

struct TrConsts {
  float l1, l2, l3;  // ln2/256 in three parts (l1 with 9 significant bits)
};

struct TrBin {
  double k0;     // smallest value
  double scale;  // 2^F
  int jz;        // values equal to k0 (they lead the sorted bin)
  int ju;        // values equal to k0 or below k0 + 2^(F-100) (FP64 terms from jz on)
  int ok;        // sorted, finite, non-negative
  int pad;
};

__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
  const float h = p + e;
  return make_float2(h, e - (h - p));
}

constexpr int TR_TAB = 256;  // 2^{-j/256}, j = 0..255

// 2^{-j/256}, j = 0..255, as float-float pairs (from FP64 exp2)
__device__ __forceinline__ void tr_table(float2 *tab) {
  for (int j = threadIdx.x; j < TR_TAB; j += blockDim.x) {
    const double t = exp2(-(double)j / (double)TR_TAB);
    const float h = (float)t;
    tab[j] = make_float2(h, (float)(t - (double)h));
  }
}

// e^{-d} for d = dh + dl in [0, 87) (|dl| <= ulp(dh)/2), as a pair:
// d = (n/256) ln 2 - r with |r| <= ln2/512, e^{-d} = 2^{-n/256} e^r,
// e^r = 1 + r + (r^2/2)(1 + r/3 + r^2/12) (truncation below 1e-18; the
// bracket's deviation from 1, < 4.6e-4, in FP32).
__device__ __forceinline__ float2 ff_exp_neg(float dh, float dl, const float2 *tab, const TrConsts &L) {
  const float n = rintf(dh * 369.32993046757458f);  // 256 / ln 2
  const int ni = (int)n;
  // r = n ln2/256 - d: n l1 is exact (l1 has 9 significant bits, n < 2^15)
  float s, e1;
  two_sum_f(n * L.l1, -dh, s, e1);
  const float b = n * L.l2;
  const float be = fmaf(n, L.l2, -b);
  float rh, e2;
  two_sum_f(s, b, rh, e2);
  float rl = ((e1 + e2) + (be - dl)) + n * L.l3;
  {
    const float t = rh + rl;
    rl = rl - (t - rh);
    rh = t;
  }
  // r^2/2 as a pair, times the bracket
  const float r2h = rh * rh;
  const float r2l = fmaf(2.0f * rh, rl, fmaf(rh, rh, -r2h));
  const float bm1 = rh * fmaf(rh, 1.0f / 12.0f, 1.0f / 3.0f);
  const float qh = 0.5f * r2h;
  const float ql = fmaf(qh, bm1, 0.5f * r2l);
  // E = r + q = e^r - 1
  float Eh, Ee;
  two_sum_f(rh, qh, Eh, Ee);
  float El = Ee + (rl + ql);
  {
    const float t = Eh + El;
    El = El - (t - Eh);
    Eh = t;
  }
  // 2^{-n/256} (1 + E) = T + T E, T = 2^{-(n & 255)/256}, then 2^{-(n >> 8)} (n >> 8 <= 125)
  const float2 T = tab[ni & (TR_TAB - 1)];
  const float2 v = ff_add(T, ff_mul(T, make_float2(Eh, El)));
  const float sc = __int_as_float((127 - (ni >> 8)) << 23);
  return make_float2(v.x * sc, v.y * sc);
}

// (sh, sl) += e, renormalized so that |sl| stays within half an ulp of sh
// (terms near 1 added to a sum near N would otherwise grow sl, and its FP32
// rounding, with every term)
__device__ __forceinline__ void tr_acc(float &sh, float &sl, float2 e) {
  float t, err;
  two_sum_f(sh, e.x, t, err);
  sl += err + e.y;
  sh = t + sl;
  sl = sl - (sh - t);
}

// d = D M as a pair (D, M pairs)
__device__ __forceinline__ float2 ff_prod(float2 D, float2 M) {
  const float h = D.x * M.x;
  const float e = fmaf(D.x, M.y, fmaf(D.y, M.x, fmaf(D.x, M.x, -h)));
  const float t = h + e;
  return make_float2(t, e - (t - h));
}

__device__ __forceinline__ float2 split_pair(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// Per bin: k_0, the scale, the counts of equal and of tiny differences, and
// the differences as scaled pairs D (one CTA per bin).
__global__ void __launch_bounds__(TR_THREADS)
    k_trans_prep(const double *__restrict__ sorted, int64_t nb, float2 *__restrict__ D, TrBin *__restrict__ bins) {
  __shared__ int s_jz, s_ju;
  const int b = blockIdx.x;
  const double *k = sorted + (int64_t)b * nb;
  const double k0 = k[0], kmax = k[nb - 1];
  if (threadIdx.x == 0) {
    s_jz = 0;
    s_ju = 0;
  }
  __syncthreads();
  bool bad = false;
  for (int64_t j = threadIdx.x; j < nb; j += TR_THREADS) {
    const double v = k[j];
    bad |= !(v >= 0.0 && isfinite(v)) || (j > 0 && !(k[j - 1] <= v));
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) bins[b] = TrBin{k0, 1.0, 0, 0, 0, 0};
    return;
  }
  const double dmax = kmax - k0;
  const int F = dmax > 0.0 ? ilogb(dmax) : 0;
  const double inv = ldexp(1.0, -F);
  const double tiny = ldexp(1.0, F - 100);
  int jz = 0, ju = 0;
  for (int64_t j = threadIdx.x; j < nb; j += TR_THREADS) {
    const double dj = k[j] - k0;
    D[(int64_t)b * nb + j] = split_pair(dj * inv);
    jz += dj == 0.0;
    ju += dj == 0.0 || dj < tiny;  // (tiny is 0 when 2^(F-100) underflows)
  }
  for (int o = 16; o > 0; o >>= 1) {
    jz += __shfl_down_sync(0xffffffffu, jz, o);
    ju += __shfl_down_sync(0xffffffffu, ju, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_jz, jz);
    atomicAdd(&s_ju, ju);
  }
  __syncthreads();
  if (threadIdx.x == 0) bins[b] = TrBin{k0, ldexp(1.0, F), s_jz, s_ju, 1, 0};
}

// The sum of the terms of one (bin, m) over the CTA, in a fixed order.
__device__ __forceinline__ double tr_block_sum(double v, double *red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < TR_THREADS / 32; ++w) t += red[w];
  return t;  // on thread 0
}

// One warp per (bin, column mass): a CTA takes one bin and TR_THREADS/32 of
// its column masses at a time (no CTA barrier); each warp finds its range of
// terms by a 32-ary search and sums them in a fixed order.
__global__ void __launch_bounds__(TR_THREADS)
    k_trans_direct(const double *__restrict__ sorted, int64_t nb, int nm, const double *__restrict__ m,
                   const float2 *__restrict__ D, const TrBin *__restrict__ bins, TrConsts L,
                   double *__restrict__ out) {
  __shared__ float2 tab[TR_TAB];
  tr_table(tab);
  __syncthreads();
  const int b = blockIdx.x, lane = threadIdx.x & 31;
  const double *k = sorted + (int64_t)b * nb;
  const float2 *Db = D + (int64_t)b * nb;
  const TrBin B = bins[b];
  constexpr int WPB = TR_THREADS / 32;
  for (int i = blockIdx.y * WPB + (threadIdx.x >> 5); i < nm; i += gridDim.y * WPB) {  // warp-uniform
    const double mi = m[i];
    double res = 0.0;
    if (!B.ok) {  // the plain FP64 sum
      double s = 0.0;
      for (int64_t j = lane; j < nb; j += 32) s += exp(-k[j] * mi);
      res = warp_sum(s) / (double)nb;
    } else {
      const double E0 = exp(-(B.k0 * mi));
      if (E0 > 0.0) {  // else every term underflows, as e^{-k_0 m} does
        // jmax: the first j >= ju with (k_j - k_0) m >= 87 (nb if none), the
        // lanes probing 32 evenly spaced places of [lo, hi) a round
        int64_t lo = B.ju, hi = nb;
        while (hi > lo) {
          const int64_t span = hi - lo;
          const int64_t step = (span + 31) >> 5;
          const int64_t p = lo + (int64_t)lane * step;
          const bool past = p < hi && (k[p] - B.k0) * mi >= TR_DMAX;
          const unsigned bal = __ballot_sync(0xffffffffu, past);
          if (step == 1) {  // every place probed: the first past one, or hi
            hi = bal ? lo + __ffs(bal) - 1 : hi;
            break;
          }
          // the first lane past (the probes increase, so all later valid ones are past too);
          // none past: the answer lies after the last valid probe
          const int64_t last = (span - 1) / step;  // lanes 0..last probe inside [lo, hi)
          if (bal) {
            const int f = __ffs(bal) - 1;
            const int64_t nhi = lo + (int64_t)f * step;
            lo = f > 0 ? lo + (int64_t)(f - 1) * step + 1 : lo;
            hi = nhi;
          } else {
            lo = lo + last * step + 1;
          }
        }
        const int64_t jmax = hi;
        double pd = 0.0;  // tiny differences, FP64
        for (int64_t j = B.jz + lane; j < min((int64_t)B.ju, jmax); j += 32) pd += exp(-((k[j] - B.k0) * mi));
        float sh = 0.0f, sl = 0.0f;
        if (jmax > B.ju) {  // then m 2^F < 87 2^100 (a pair)
          const float2 M = split_pair(mi * B.scale);
          // two terms a lane per pass (independent exponentials side by side)
          int64_t j = B.ju + lane;
          for (; j + 32 < jmax; j += 64) {
            const float2 d0 = ff_prod(Db[j], M), d1 = ff_prod(Db[j + 32], M);
            const float2 e0 = ff_exp_neg(fminf(d0.x, 86.0f), d0.y, tab, L);
            const float2 e1 = ff_exp_neg(fminf(d1.x, 86.0f), d1.y, tab, L);
            if (d0.x < (float)TR_DMAX) tr_acc(sh, sl, e0);
            if (d1.x < (float)TR_DMAX) tr_acc(sh, sl, e1);
          }
          if (j < jmax) {
            const float2 d = ff_prod(Db[j], M);
            if (d.x < (float)TR_DMAX) tr_acc(sh, sl, ff_exp_neg(d.x, d.y, tab, L));
          }
        }
        const double t = warp_sum((double)sh + (double)sl + pd);
        res = E0 * ((double)B.jz + t) / (double)nb;
      }
    }
    if (lane == 0) out[(int64_t)b * nm + i] = res;
  }
}

// k(g) of a bin from its fit at g_j = (j + 1/2)/ng, FP64
__device__ __forceinline__ double tr_kfit(const double *c, int ncheb, int j, int ng) {
  const double t = 2.0 * (((double)j + 0.5) / (double)ng) - 1.0;
  double tkm1 = 1.0, tk = t, v = c[0];
  if (ncheb > 1) v += c[1] * t;
  for (int q = 2; q < ncheb; ++q) {
    const double tn = 2.0 * t * tk - tkm1;
    v += c[q] * tn;
    tkm1 = tk;
    tk = tn;
  }
  return exp(v);
}

// One CTA per (bin, block of column masses), one column mass a thread, the
// fit's ng values of k (and their pairs) in shared memory.  The values are
// not sorted, so every point is visited; terms with d >= 87 are skipped.
__global__ void __launch_bounds__(TR_THREADS)
    k_trans_fit(const double *__restrict__ coef, int ncheb, int ng, int nm, const double *__restrict__ m,
                TrConsts L, double *__restrict__ out) {
  extern __shared__ double kfit[];  // ng values, then ng pairs (a negative pair: FP64 term)
  float2 *Dg = reinterpret_cast<float2 *>(kfit + ng);
  __shared__ float2 tab[TR_TAB];
  __shared__ double rmin[TR_THREADS / 32], rmax[TR_THREADS / 32];
  tr_table(tab);
  const int b = blockIdx.x;
  const double *c = coef + (int64_t)b * ncheb;
  double vmin = INFINITY, vmax = 0.0;
  bool bad = false;
  for (int j = threadIdx.x; j < ng; j += TR_THREADS) {
    const double v = tr_kfit(c, ncheb, j, ng);
    kfit[j] = v;
    bad |= !isfinite(v);
    vmin = fmin(vmin, v);
    vmax = fmax(vmax, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    vmin = fmin(vmin, __shfl_down_sync(0xffffffffu, vmin, o));
    vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    rmin[threadIdx.x >> 5] = vmin;
    rmax[threadIdx.x >> 5] = vmax;
  }
  bad = __syncthreads_or(bad);
  vmin = INFINITY;
  vmax = 0.0;
  for (int w = 0; w < TR_THREADS / 32; ++w) {
    vmin = fmin(vmin, rmin[w]);
    vmax = fmax(vmax, rmax[w]);
  }
  const double dmax = vmax - vmin;
  const int F = dmax > 0.0 ? ilogb(dmax) : 0;
  const double inv = ldexp(1.0, -F), tiny = ldexp(1.0, F - 100), scale = ldexp(1.0, F);
  if (!bad)
    for (int j = threadIdx.x; j < ng; j += TR_THREADS) {
      const double dj = kfit[j] - vmin;
      Dg[j] = (dj == 0.0 || dj >= tiny) ? split_pair(dj * inv) : make_float2(-1.0f, 0.0f);
    }
  __syncthreads();
  for (int i = blockIdx.y * TR_THREADS + threadIdx.x; i < nm; i += gridDim.y * TR_THREADS) {
    const double mi = m[i];
    double res;
    if (bad) {  // the plain FP64 sum
      double s = 0.0;
      for (int j = 0; j < ng; ++j) s += exp(-kfit[j] * mi);
      res = s / (double)ng;
    } else {
      const double E0 = exp(-(vmin * mi));
      res = 0.0;
      if (E0 > 0.0) {
        const double Md = mi * scale;
        const bool pairs = Md < 0x1p107;  // else every pair term has d >= 128
        const float2 M = split_pair(pairs ? Md : 0.0);
        float sh = 0.0f, sl = 0.0f;
        double pd = 0.0;
        for (int j = 0; j < ng; ++j) {
          const float2 Dj = Dg[j];
          if (Dj.x < 0.0f) {
            pd += exp(-((kfit[j] - vmin) * mi));
          } else if (pairs) {
            const float2 d = ff_prod(Dj, M);
            if (d.x < (float)TR_DMAX) {
              tr_acc(sh, sl, ff_exp_neg(d.x, d.y, tab, L));
            }
          }
        }
        res = E0 * ((double)sh + (double)sl + pd) / (double)ng;
      }
    }
    out[(int64_t)b * nm + i] = res;
  }
}

// The plain FP64 fit transmission, for ng too large for k_trans_fit's shared
// memory (16 B a point).
__global__ void __launch_bounds__(TR_THREADS)
    k_trans_fit64(const double *__restrict__ coef, int ncheb, int ng, int nm, const double *__restrict__ m,
                double *__restrict__ out) {
  extern __shared__ double kfit[];  // ng values
  const int b = blockIdx.x;
  const double *c = coef + (int64_t)b * ncheb;
  for (int j = threadIdx.x; j < ng; j += TR_THREADS) {
    const double t = 2.0 * (((double)j + 0.5) / (double)ng) - 1.0;
    double tkm1 = 1.0, tk = t, v = c[0];
    if (ncheb > 1) v += c[1] * t;
    for (int q = 2; q < ncheb; ++q) {
      const double tn = 2.0 * t * tk - tkm1;
      v += c[q] * tn;
      tkm1 = tk;
      tk = tn;
    }
    kfit[j] = exp(v);
  }
  __syncthreads();
  for (int i = blockIdx.y * TR_THREADS + threadIdx.x; i < nm; i += gridDim.y * TR_THREADS) {
    const double mi = m[i];
    double s = 0.0;
    for (int j = 0; j < ng; ++j) s += exp(-kfit[j] * mi);
    out[(int64_t)b * nm + i] = s / (double)ng;
  }
}

// ln2/256 in three parts, the first with 9 significant bits (so that n l1 is
// exact for n < 2^15)
static TrConsts tr_consts() {
  const double L = 0.69314718055994530941723212145817657 / 256.0;
  float l1 = (float)L;
  uint32_t u;
  memcpy(&u, &l1, 4);
  u &= 0xFFFF8000u;
  memcpy(&l1, &u, 4);
  const float l2 = (float)(L - (double)l1);
  const float l3 = (float)(L - (double)l1 - (double)l2);
  return TrConsts{l1, l2, l3};
}

size_t trans_pair_bytes(int nbins, int64_t nb) { return (size_t)nbins * (size_t)nb * sizeof(float2); }
size_t trans_bin_bytes(int nbins) { return (size_t)nbins * sizeof(TrBin); }

cudaError_t launch_transmission(helk_ctx *c, int nbins, int64_t nb, const double *sorted,
                                const double *coef, int ncheb, int ng, int nm, const double *m_dev,
                                double *direct, double *fit) {
  const TrConsts L = tr_consts();
  if (sorted && direct) {
    float2 *D = reinterpret_cast<float2 *>(c->tr_pairs);
    TrBin *bins = reinterpret_cast<TrBin *>(c->tr_bins);
    ++c->launches;
    k_trans_prep<<<nbins, TR_THREADS, 0, c->stream>>>(sorted, nb, D, bins);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid(nbins, std::max(1, std::min(8, (nm + TR_THREADS / 32 - 1) / (TR_THREADS / 32))));
    ++c->launches;
    k_trans_direct<<<grid, TR_THREADS, 0, c->stream>>>(sorted, nb, nm, m_dev, D, bins, L, direct);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (coef && fit) {
    dim3 grid(nbins, (nm + TR_THREADS - 1) / TR_THREADS);
    const size_t smem = (size_t)ng * (sizeof(double) + sizeof(float2));
    if (smem + 2048 <= (size_t)c->max_smem_optin) {
      if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_trans_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      ++c->launches;
      k_trans_fit<<<grid, TR_THREADS, smem, c->stream>>>(coef, ncheb, ng, nm, m_dev, L, fit);
    } else {
      const size_t smem64 = (size_t)ng * sizeof(double);
      if (smem64 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_trans_fit64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem64);
        if (e != cudaSuccess) return e;
      }
      ++c->launches;
      k_trans_fit64<<<grid, TR_THREADS, smem64, c->stream>>>(coef, ncheb, ng, nm, m_dev, fit);
    }
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ------------------------------------------------ allocation-free variant --
// Scratch of helk_kdist_static in a file-scope device array instead of
// cudaMalloc'd memory: the pseudo-inverse of the Chebyshev basis (N_b x
// n_cheb doubles), the Householder work array of the same size, the
// logarithm's table, and the (N_b, n_cheb) the pseudo-inverse was built for
// (zero until the first build, so never equal to a valid pair).
// Bins are limited to KDIST_STATIC_NB_MAX points (their sort then runs in
// shared memory, so no other scratch is needed) and n_cheb to NCHEB_MAX:
// 2 x 12288 x 32 x 8 B = 6 MiB, held by every device that loads the library
// until the process exits.
constexpr int64_t KDIST_STATIC_NB_MAX = 12288;
static_assert(KDIST_STATIC_NB_MAX <= KD_REG_MAX, "the static path's bins fit the register radix passes");
constexpr int64_t KDIST_STATIC_PINV = KDIST_STATIC_NB_MAX * NCHEB_MAX;
constexpr int64_t KDIST_STATIC_TAG = 2 * KDIST_STATIC_PINV + KD_LNTAB;  // offset of the size tag
static __device__ __align__(256) double g_kdist_scratch[KDIST_STATIC_TAG + 2];

namespace {
constexpr int KDIST_STATIC_MAX_DEVICES = 64;
double *g_static_ptr[KDIST_STATIC_MAX_DEVICES];  // device address of g_kdist_scratch per device
std::mutex g_static_mu;
}  // namespace

}  // namespace helk

extern "C" helk_status helk_kdist_static(const double *kappa, int64_t n, int32_t nbins,
                                         int32_t ncheb, double kappa_floor, double *coeffs,
                                         double *mean, double *kg_out, void *stream) {
  using namespace helk;
  if (!kappa || !coeffs) return HELK_ERR_INVALID_ARG;
  if (n <= 0 || nbins <= 0 || n % nbins) return HELK_ERR_INVALID_ARG;
  const int64_t nb = n / nbins;
  if (nb > KDIST_STATIC_NB_MAX || ncheb < 1 || ncheb > NCHEB_MAX || ncheb > nb)
    return HELK_ERR_INVALID_ARG;
  if (!(kappa_floor > 0.0) || !isfinite(kappa_floor)) return HELK_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= KDIST_STATIC_MAX_DEVICES) {
    cudaGetLastError();
    return HELK_ERR_CUDA;
  }
  int smem_optin = 0;
  if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return HELK_ERR_CUDA;
  const size_t smem = (size_t)nb * 16;
  if ((int64_t)smem + 26 * 1024 > smem_optin) return HELK_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double *ptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      // once per device, with that device current: the array's device address
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_kdist_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return HELK_ERR_CUDA;
      }
      g_static_ptr[dev] = (double *)p;
    }
    ptr = g_static_ptr[dev];
  }
  // The pseudo-inverse for these sizes: rebuilt on the device only when the
  // sizes recorded in the array differ (the check runs in stream order, so
  // it sees what earlier calls on the stream left there).
  k_pinv<<<1, PI_THREADS, 0, st>>>(nb, ncheb, ptr + KDIST_STATIC_PINV, nullptr, ptr,
                                   reinterpret_cast<float2 *>(ptr + 2 * KDIST_STATIC_PINV),
                                   reinterpret_cast<long long *>(ptr + KDIST_STATIC_TAG));
  if (cudaGetLastError() != cudaSuccess) return HELK_ERR_CUDA;
  if (cudaFuncSetAttribute(k_kdist_bin<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return HELK_ERR_CUDA;
  }
  k_kdist_bin<0, true><<<nbins, KD_THREADS, smem, st>>>(kappa, (int)nb, ncheb, kappa_floor,
                                                  reinterpret_cast<const float2 *>(ptr),
                                                  reinterpret_cast<const float2 *>(ptr + 2 * KDIST_STATIC_PINV),
                                                  nullptr, nullptr, coeffs, mean, kg_out, nullptr);
  return cudaGetLastError() == cudaSuccess ? HELK_OK : HELK_ERR_CUDA;
}
