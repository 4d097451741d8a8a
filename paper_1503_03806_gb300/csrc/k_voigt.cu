// k_voigt.cu -- the FP32 form of the line-tiled Voigt opacity kernel
// (Sec. 2.3-2.4): FP32 profile evaluation on records with strengths scaled by
// 2^-E, Kahan-compensated FP32 accumulation per point, the result converted
// to FP64 and rescaled at the flush; its Algorithm 916 cores in a separate
// kernel that runs beside it on a second stream; the table of kernel shapes
// the autotuner times; and the precision dispatch of the Voigt launch.
// Persistent CTAs; warp w of a tile owns 32 NSLOT consecutive grid points;
// the candidate lines of successive tiles stream through a shared-memory
// ring filled by 1-D bulk copies (see the pipeline below).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "helk_internal.cuh"
#include "voigt_common.cuh"
#include "voigt_core.cuh"

namespace helk {

// ------------------------------------------------------------ FP32 form --
// Method classes of one (line, tile) pair.  |u| is monotone in |i - c| in
// the FP32 arithmetic used per point (u = fma(d, beta, -phi) is correctly
// rounded, so monotone in the exact integer d, and fma(u, u, a^2) is monotone
// in |u|), so the extreme r^2 over the tile's covered points decide whether
// every point of the pair uses the same method.  Pure pairs run a
// branch-free loop over all slots (independent chains the compiler can
// interleave); mixed pairs -- those containing a method boundary or the line
// core -- decide per point.
enum { CLS_GH1 = 1, CLS_GH3 = 2, CLS_MIXED = 3 };  // 0: the line misses the warp
constexpr int KAHAN_GROUP = 32;             // lines per compensated partial

// Whether a core evaluation at (x, y) lies in a cell where the surrogate
// network was validated (features as in k_mlp.cu).
// The routing decision is split into a per-line part (the row of validated
// cells for y = a, or -1 when a is outside the network's range) and a
// per-point part (the column of x = |u|), both as in the network's features.
__device__ __forceinline__ int surr_row(const SurrQueue *sq, float y) {
  if (!sq || !(y >= 1.0e-4f && y < 10.0f)) return -1;
  const float f2 = 0.4f * (log10f(y) + 4.0f) - 1.0f;
  const int cy = min(max((int)((f2 + 1.0f) * 0.5f * sq->ny), 0), sq->ny - 1);
  return cy * sq->nx;
}

__device__ __forceinline__ bool surr_route(const SurrQueue *sq, int row, float x) {
  const float f1 = 2.0f * asinhf(x) * (float)(1.0 / ASINH_XCORE) - 1.0f;
  const int cx = min(max((int)((f1 + 1.0f) * 0.5f * sq->nx), 0), sq->nx - 1);
  const int cell = row + cx;
  return (sq->mask[cell >> 5] >> (cell & 31)) & 1u;
}

// One queue slot per calling lane: the lanes that arrive together take one
// atomicAdd for all of them (a single counter would otherwise see one atomic
// per routed evaluation).
__device__ __forceinline__ unsigned long long surr_reserve(SurrQueue *sq) {
  namespace cg = cooperative_groups;
  const cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&sq->count, (unsigned long long)g.size());
  return g.shfl(base, 0) + g.thread_rank();
}

// One core evaluation (x^2 + y^2 < 100): S' K by Algorithm 916, or 0 after
// appending the point to the surrogate's queue when its cell is validated
// (the queue's kernel adds it later).
__device__ __forceinline__ float core_point(const LineRec32 &L, float x, int i, int srow, SurrQueue *sq,
                                         int cond, const float *w) {
  if (srow >= 0 && surr_route(sq, srow, x)) {
    const unsigned long long slot = surr_reserve(sq);
    if (slot < sq->cap) {
      sq->idx[slot] = i;
      sq->cond[slot] = cond;
      sq->w[slot] = L.Sp;
      sq->x[slot] = x;
      sq->y[slot] = L.a;
      return 0.0f;
    }
  }
  return L.Sp * k916_f32(x, L.a, L.erfcx_a, L.sig1, w);
}

// Hardware reciprocal approximation (max relative error ~1 ulp); every
// argument here is >= 100, far from the denormal range.
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// v 2^E as a double, for a normal float v, from its bits (integer
// operations only: the conversion and scaling would otherwise be two
// operations of the FP64 unit, which runs at 1/64 of the FP32 rate here).
// Exact: the double holds v's sign and 24-bit significand at the shifted
// exponent; zero stays (signed) zero.  A subnormal v, or a result outside
// the double's normal range, takes the FP64 route.
__device__ __forceinline__ double scaled_to_double(float v, int E) {
  const unsigned b = __float_as_uint(v);
  if ((b & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)((unsigned long long)(b >> 31) << 63));
  const int ef = (int)((b >> 23) & 0xFF);
  const int e = ef - 127 + 1023 + E;
  if (ef == 0 || e <= 0 || e >= 2047) return ldexp((double)v, E);
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)e << 52) |
                                          ((unsigned long long)(b & 0x7FFFFF) << 29)));
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Kahan-adds the plain partials into (sum, comp) and starts a new group.
// The loops over a group's lines run in stretches that end where the group
// is full, so the check is made once per stretch, not once per line.
template <int NSLOT>
__device__ __forceinline__ void kahan_fold(int &ngroup, float (&sum)[NSLOT], float (&comp)[NSLOT],
                                           float (&part)[NSLOT]) {
  ngroup = 0;
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    kahan_add(sum[k], comp[k], part[k]);
    part[k] = 0.0f;
  }
}

// 3-node Gauss-Hermite (nodes 0, +-t, t^2 = 3/2, weights 4 w1, w1):
//   (a w1/pi) [4/r2 + 2q/p],  q = r2 + t^2,  p = ((u-t)^2+a^2)((u+t)^2+a^2).
// With u^2 = r2 - a^2 both factors are polynomials in r2 alone:
//   p = r2 (r2 - 3) + C,  C = 9/4 + 6 a^2,
//   2p + q r2 = r2 (3 r2 - 9/2) + 2C,
// so the term is n / (r2 p) with n = r2 (c3 r2 + c45) + c2, the line's
// factor P3h = 2 a w1 S'/pi folded into c3 = 3 P3h, c45 = -9/2 P3h,
// c2 = 2C P3h.  No cancellation for r2 >= 100 (r2^2 >= 33 x 3 r2); FP32
// relative error < 5e-7 over 100 <= r2 < 1e6.
struct Gh3Line {
  float a2, C, c3, c45, c2;
  Gh3Line() = default;
  __device__ __forceinline__ Gh3Line(float a2_, float C_, float c3_, float c45_, float c2_)
      : a2(a2_), C(C_), c3(c3_), c45(c45_), c2(c2_) {}
  __device__ __forceinline__ Gh3Line(float a2_, float P3) {
    const float P3h = 2.0f * P3;
    a2 = a2_;
    C = fmaf(6.0f, a2_, 2.25f);
    c3 = 3.0f * P3h;
    c45 = -4.5f * P3h;
    c2 = P3h * fmaf(12.0f, a2_, 4.5f);
  }
  // numerator and denominator of the term, for the point's r2 = u^2 + a^2
  __device__ __forceinline__ void nd(float r2, float &n, float &d) const {
    const float p = fmaf(r2, r2 - 3.0f, C);
    n = fmaf(r2, fmaf(c3, r2, c45), c2);
    d = r2 * p;
  }
  // part + term
  __device__ __forceinline__ float add(float part, float r2) const {
    float n, d;
    nd(r2, n, d);
    return fmaf(n, fast_rcp(d), part);
  }
};

// The same term far from the line centre as a series in t = 1/r2:
//   n / (r2 p) = t (c3 + c45 t + c2 t^2) / (1 - 3 t + C t^2)
//              = t (g0 + g1 t + g2 t^2 + g3 t^3 + ...),
//   g0 = 3 P3h, g1 = 4.5 P3h, g2 = (11.25 - 6 a^2) P3h, g3 = (23.625 - 45 a^2) P3h
// (the product of the numerator's coefficients with those of 1/(1 - 3t +
// C t^2), e_0 = 1, e_1 = 3, e_k = 3 e_{k-1} - C e_{k-2}).  Truncated after g2,
// on r2 >= R_s with R_s >= 1000 and R_s^3 >= 1.25^3 5e7 (7.875 + 15 a^2)
// (>= 1.25^3 5e7 |g3/g0|), the relative truncation error is below 1.1e-8 for
// every a (checked in FP64 on a grid of a^2 in [0, 1e6) and r2 in [R_s, 1e6)),
// under the FP32 rounding of either form: one reciprocal and three FMAs
// instead of five FP32 operations and one reciprocal.
struct Gh3Series {
  float g0, g1, g2;
  __device__ __forceinline__ explicit Gh3Series(float a2, float P3) {
    const float P3h = 2.0f * P3;
    g0 = 3.0f * P3h;
    g1 = 4.5f * P3h;
    g2 = P3h * fmaf(-6.0f, a2, 11.25f);
  }
  // does the series hold on a span whose smallest r2 is r2near?
  static __device__ __forceinline__ bool holds(float r2near, float a2) {
    return r2near >= 1000.0f && r2near * r2near * r2near >= 9.765625e7f * fmaf(15.0f, a2, 7.875f);
  }
};

// ---- FP32 line pipeline: a ring of F32_STAGES chunks of candidate lines,
// filled by 1-D bulk copies that complete on the stage's mbarrier, with no
// CTA-wide barrier in the main loop.  Every warp consumes the chunk stream in
// order; the warp that finishes a chunk last (a shared-memory counter per
// stage) refills that stage with the chunk F32_STAGES further on, fetching
// the next (condition, tile) item from the global counter when the current
// one has no lines left.  So warps may drift apart by several chunks instead
// of meeting at a barrier after each one.  Each chunk carries a header (item,
// first line, count); an item without lines gets one empty chunk so that its
// tile is still written, and an exhausted item counter ends the stream with
// an empty chunk of item -1.
constexpr int F32_STAGES = 5;

struct ChunkHdr {
  int item, l0, cnt, pad;
};

struct F32Pipe {
  ChunkHdr hdr[F32_STAGES];
  unsigned long long full[F32_STAGES];
  int done[F32_STAGES];
  int pending[F32_STAGES];  // parity + 1 of a copy in flight into the stage, else 0
  int item, pos, end, exhausted;  // the issuer's place in the stream
};

// Publishes chunk `seq` of the stream into stage seq % F32_STAGES.  Called by
// one thread at a time (the initial fill, then the last consumer of the chunk
// that used the stage before).
template <int LCH>
__device__ void f32_issue(F32Pipe &P, LineRec32 (*sl)[LCH], unsigned long long seq, const LineRec32 *rec_all,
                          int64_t nlines, const int32_t *tlo_all, const int32_t *thi_all, int64_t ntiles,
                          const int *cond_order, int nitems, DevStats *st) {
  const int s = (int)(seq % F32_STAGES);
  const uint32_t mb = smem_addr(&P.full[s]);
  if (P.item < 0 || P.pos >= P.end) {  // the current item has no lines left: take the next one
    int item = -1;
    if (!P.exhausted) {
      item = (int)atomicAdd(&st->tile_counter, 1u);
      if (item >= nitems) item = -1;
    }
    if (item < 0) {
      P.exhausted = 1;
      P.hdr[s] = ChunkHdr{-1, 0, 0, 0};
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
      return;
    }
    const int cond = cond_order[item / ntiles];
    const int64_t t = (int64_t)cond * ntiles + item % ntiles;
    P.item = item;
    P.pos = tlo_all[t];
    P.end = thi_all[t];
    if (P.pos >= P.end) {
      P.hdr[s] = ChunkHdr{item, P.pos, 0, 0};
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
      return;
    }
  }
  const int cnt = min(LCH, P.end - P.pos);
  const int cond = cond_order[P.item / ntiles];
  P.hdr[s] = ChunkHdr{P.item, P.pos, cnt, 0};
  P.pending[s] = (int)((seq / F32_STAGES) & 1ull) + 1;
  // the stage's previous contents were read through the generic proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tma_load_1d(smem_addr(&sl[s][0]), rec_all + (int64_t)cond * nlines + P.pos,
              (uint32_t)(cnt * sizeof(LineRec32)), mb);
  P.pos += cnt;
}

// After a failed wait: wait (bounded) for the copies still in flight, so that
// none lands in shared memory after the CTA has left.
__device__ void f32_drain(F32Pipe &P, int *flags) {
  for (int s = 0; s < F32_STAGES; ++s) {
    const int pend = *((volatile int *)&P.pending[s]);
    if (pend) mbar_wait_bounded(smem_addr(&P.full[s]), (uint32_t)(pend - 1), flags, WAIT_LIMIT_NS);
  }
}

// What one warp needs of one line, prepared by one lane (lanes in parallel)
// and read by the whole warp with three broadcast loads: the kind of the
// (line, warp) pair, the covered points, the point offset, and the method's
// constants.
//   Whole-span lines (one method on every point of the warp's span: GH1, or
//   GH3 by its expansion in 1/r^2 (Gh3Series) where that holds on the whole
//   span, r^2 >= R_s; the line centre outside the span): u is stepped from the span edge
//   nearest the centre, u_k = fma(k - k_b, 32 beta, u_b), one FMA a slot (the
//   step product is exact, so each u_k is rounded once and |u_b| <= |u_k|
//   bounds its error by one ulp of u_k); d0 = (float)(base point - c) of lane
//   0, k_b = 0 (kind *_FWD, centre at or before the span) or NSLOT - 1
//   (*_BWD, centre at or after it).
//   The rest (partial cover, a method boundary, the core, the centre inside
//   the span, or GH3 nearer the centre than R_s, where the term is formed
//   exactly): d0 = (float)(wbase - c) and u = (d0 + lane + 32 k) beta
//   - phi with d0 + lane + 32 k exact, so every point's method (and whether
//   it is a core point, left to the core kernel) is decided on the same
//   correctly rounded u as in k_core_f32.
//   The series covers most of the GH3 region; the GH3 spans nearer the
//   centre run as the rest rather than in a whole-span loop of their own
//   (with one loop kind fewer the main loop's code stays within the
//   instruction caches: 0.743 against 0.763 ms a medium step).
enum { KIND_MISS = 0, KIND_GH1_FWD = 1, KIND_GH1_BWD = 2, KIND_GH3S_FWD = 3, KIND_GH3S_BWD = 4, KIND_REST = 5 };
constexpr int NKIND = 5;  // kinds after KIND_MISS

struct __align__(16) WarpLine {
  int kind;          // KIND_*
  int cls;           // CLS_* (KIND_REST)
  int lo, hi;        // covered points (grid indices; KIND_REST)
  float d0;          // point offset of lane 0 at the base slot (see above)
  float beta, nphi, a2;
  float q0, q1, q2, q3;  // GH1: P1; GH3S: g0, g1, g2 (Gh3Series); rest: P1, or GH3's C, c3, c45, c2 (Gh3Line)
};

// Whole-span lines [t, t1) of one kind: GH1 or GH3 by its series, u stepped
// from the base slot.  GH1 takes one reciprocal for two slots, 1/r_a^2 =
// r_b^2 / (r_a^2 r_b^2) (5 instructions and half a reciprocal an evaluation
// instead of 4 and one: the MUFU unit, at 16 reciprocals a clock per SM, is
// the co-bound of this loop mix); the series keeps one reciprocal a slot (6
// instructions), where pairing would make the issue count the bound.
template <int NSLOT, bool FWD, bool GH3S>
__device__ __forceinline__ void span_lines(const WarpLine *wl, int t, int t1, float lanef, int &ngroup,
                                           float (&sum)[NSLOT], float (&comp)[NSLOT], float (&part)[NSLOT]) {
  while (t < t1) {
    const int te = min(t1, t + KAHAN_GROUP - ngroup);
    ngroup += te - t;
    for (; t < te; ++t) {
      const WarpLine &W = wl[t];
      const float beta = W.beta, a2 = W.a2;
      const float ub = fmaf(W.d0 + lanef, beta, W.nphi);  // u at the base slot
      const float h = 32.0f * beta;                        // u step between slots (exact)
      if (GH3S) {
        const float g0 = W.q0, g1 = W.q1, g2 = W.q2;
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
          const float u = fmaf(FWD ? (float)k : (float)(k - (NSLOT - 1)), h, ub);
          const float rr = fast_rcp(fmaf(u, u, a2));  // t = 1/r^2 of the series
          part[k] = fmaf(rr, fmaf(fmaf(g2, rr, g1), rr, g0), part[k]);
        }
      } else {
        const float P1 = W.q0;
#pragma unroll
        for (int k = 0; k + 1 < NSLOT; k += 2) {
          const float u0 = fmaf(FWD ? (float)k : (float)(k - (NSLOT - 1)), h, ub);
          const float u1 = fmaf(FWD ? (float)(k + 1) : (float)(k + 1 - (NSLOT - 1)), h, ub);
          const float ra = fmaf(u0, u0, a2), rb = fmaf(u1, u1, a2);
          const float rr = fast_rcp(ra * rb);
          part[k] = fmaf(P1 * rb, rr, part[k]);
          part[k + 1] = fmaf(P1 * ra, rr, part[k + 1]);
        }
        if (NSLOT & 1) {
          const float u = fmaf(FWD ? (float)(NSLOT - 1) : 0.0f, h, ub);
          part[NSLOT - 1] = fmaf(P1, fast_rcp(fmaf(u, u, a2)), part[NSLOT - 1]);
        }
      }
    }
    if (ngroup == KAHAN_GROUP) kahan_fold<NSLOT>(ngroup, sum, comp, part);
  }
}

// MINB resident CTAs per SM: 3 (<= 85 registers a thread) or 2.
template <int BLOCK, int NSLOT, int LCH, bool COUNT, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
    k_voigt_f32(const LineRec32 *__restrict__ rec_all, int64_t nlines,
                const int32_t *__restrict__ tlo_all, const int32_t *__restrict__ thi_all,
                int64_t ntiles, const int *__restrict__ cond_order, int n_cond, int ngrid,
                double weight, int accumulate, double *__restrict__ kappa_all, CondStats *cst,
                DevStats *st, SurrQueue *sq) {
  // Warp w of the CTA owns the WSPAN consecutive points starting at
  // base + w WSPAN; lane l holds points base + w WSPAN + 32 k + l.  Method
  // classes are decided per (line, warp), so only the warps whose span holds
  // a method boundary or the line core take the per-point path.
  constexpr int NW = BLOCK / 32;
  constexpr int TILE = BLOCK * NSLOT;
  constexpr int WSPAN = 32 * NSLOT;
  constexpr int LPL = LCH / 32;  // lines of a chunk per lane in the class pass
  static_assert(LCH % 32 == 0 && LPL * 3 <= 32, "3 class bits per line in one word");
  __shared__ __align__(128) LineRec32 sl[F32_STAGES][LCH];
  __shared__ __align__(8) F32Pipe P;
  __shared__ WarpLine s_wl[NW][32];
  const int lane = threadIdx.x & 31;
  const int nitems = (int)(ntiles * n_cond);
  if (threadIdx.x == 0) {
    for (int s = 0; s < F32_STAGES; ++s) {
      mbar_init(smem_addr(&P.full[s]), 1);
      P.done[s] = 0;
      P.pending[s] = 0;
    }
    P.item = -1;
    P.pos = P.end = 0;
    P.exhausted = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (unsigned long long q = 0; q < F32_STAGES; ++q)
      f32_issue<LCH>(P, sl, q, rec_all, nlines, tlo_all, thi_all, ntiles, cond_order, nitems, st);

  // cur: the item being accumulated; -2 before the first chunk (-1 marks the
  // end of the stream, so a CTA that gets no item at all still sees a change)
  int cur = -2, wbase = 0;
  // No stream is longer than every item's chunks plus the end markers: a
  // longer one means a logic error, reported instead of looping.
  const uint32_t max_seq = (uint32_t)min(
      (unsigned long long)nitems * (unsigned long long)(nlines / LCH + 2) + 2 * F32_STAGES, 0x7FFFFFFFull);
  // Compensated accumulation: each point sums KAHAN_GROUP lines plainly
  // into part[k] (relative error <= 31 u, all terms positive) and Kahan-adds
  // the partial into (sum, comp); total relative error < 2e-6.
  float sum[NSLOT], comp[NSLOT], part[NSLOT];
  int ngroup = 0;
  unsigned long long cnt[4] = {0, 0, 0, 0};
  for (uint32_t seq = 0;; ++seq) {
    const int s = (int)(seq % F32_STAGES);
    if (seq > max_seq) {
      if (lane == 0) {
        atomicOr(&st->err_flags, ERRF_TIMEOUT);
        f32_drain(P, &st->err_flags);
      }
      return;
    }
    if (!mbar_wait_bounded(smem_addr(&P.full[s]), (seq / F32_STAGES) & 1u, &st->err_flags, WAIT_LIMIT_NS)) {
      if (lane == 0) f32_drain(P, &st->err_flags);
      return;
    }
    const ChunkHdr h = P.hdr[s];
    if (h.item != cur) {
      if (cur >= 0) {  // the previous tile is complete: write it
        const int cond = cond_order[cur / ntiles];
        double *kappa = kappa_all + (int64_t)cond * ngrid;
        const int E = cst[cond].scale_exp;
        const double scale = ldexp(weight, E);
        const bool unit = weight == 1.0;
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
          kahan_add(sum[k], comp[k], part[k]);
          const int i = wbase + lane + 32 * k;
          if (i < ngrid) {
            // 2^E (sum - comp): for weight 1 the two scaled values are formed on
            // the integer pipe (exact) and one FP64 subtraction rounds, the
            // same result as scaling the FP64 difference
            const double v = unit ? scaled_to_double(sum[k], E) - scaled_to_double(comp[k], E)
                                  : scale * ((double)sum[k] - (double)comp[k]);
            kappa[i] = accumulate ? kappa[i] + v : v;
          }
        }
        if (COUNT) {
          for (int r = 0; r < 4; ++r) {
            unsigned long long v = cnt[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(&cst[cond].region[r], v);
            cnt[r] = 0;
          }
        }
      }
      if (h.item < 0) return;  // end of the stream
      cur = h.item;
      wbase = (int)((cur % ntiles) * TILE) + (threadIdx.x >> 5) * WSPAN;
#pragma unroll
      for (int k = 0; k < NSLOT; ++k) {
        sum[k] = 0.0f;
        comp[k] = 0.0f;
        part[k] = 0.0f;
      }
      ngroup = 0;
    }
    if (lane == 0) P.pending[s] = 0;
    const LineRec32 *buf = sl[s];
    const int cnum = h.cnt;
    // The chunk in groups of 32 lines: lane l prepares line 32 m + l for this
    // warp (method class: the extreme r^2 over the warp's covered points
    // [lo, hi] decides it, r^2(d) being monotone on each side of the line
    // centre in the FP32 arithmetic of the evaluation loops), then the warp
    // runs through the group.
    WarpLine *wl = s_wl[threadIdx.x >> 5];
    const float lanef = (float)lane;
    for (int m0 = 0; m0 < cnum; m0 += 32) {
    int nk[NKIND];  // first record of each kind after KIND_GH1_FWD, in kind order
    {
      const int j = m0 + lane;
      WarpLine r;
      r.kind = KIND_MISS;
      if (j < cnum) {
        const LineRec32 &L = buf[j];
        const int c = L.c;
        const int lo = max(L.ilo, wbase), hi = min(L.ihi, wbase + WSPAN - 1);
        if (lo <= hi) {
          const float beta = L.beta, nphi = -L.phi_k, a2 = L.a2;
          const int dlo = lo - c, dhi = hi - c;
          const int dnear = dlo >= 1 ? dlo : (dhi <= -1 ? dhi : 0);
          const float un = fmaf((float)dnear, beta, nphi);
          const float ul = fmaf((float)dlo, beta, nphi), uh = fmaf((float)dhi, beta, nphi);
          const float r2near = fmaf(un, un, a2);
          const float r2far = fmaxf(fmaf(ul, ul, a2), fmaf(uh, uh, a2));
          const int cls = r2near >= 1.0e6f ? CLS_GH1
                                           : ((r2near >= 100.0f && r2far < 1.0e6f) ? CLS_GH3 : CLS_MIXED);
          const bool full = (lo == wbase) && (hi == wbase + WSPAN - 1);
          r.cls = cls;
          r.lo = lo;
          r.hi = hi;
          r.beta = beta;
          r.nphi = nphi;
          r.a2 = a2;
          const bool series = cls == CLS_GH3 && Gh3Series::holds(r2near, a2);
          // (GH1 spans reach r^2 < 1e18 only: the paired reciprocals' product
          // of two r^2 stays inside the FP32 range; farther spans run as the rest)
          if (full && ((cls == CLS_GH1 && r2far < 1.0e18f) || series) && (dlo >= 0 || dhi <= 0)) {
            const bool fwd = dlo >= 0;
            r.kind = (cls == CLS_GH1 ? KIND_GH1_FWD : KIND_GH3S_FWD) + (fwd ? 0 : 1);
            r.d0 = (float)(fwd ? dlo : dhi - 31);  // lane 0 at slot 0 or NSLOT - 1
          } else {
            r.kind = KIND_REST;
            r.d0 = (float)(wbase - c);
          }
          if (series && r.kind != KIND_REST) {
            const Gh3Series gs(a2, L.P3);
            r.q0 = gs.g0;
            r.q1 = gs.g1;
            r.q2 = gs.g2;
          } else if (cls == CLS_GH3) {
            const Gh3Line g3(a2, L.P3);
            r.q0 = g3.C;
            r.q1 = g3.c3;
            r.q2 = g3.c45;
            r.q3 = g3.c2;
          } else {
            r.q0 = L.P1;
          }
        }
      }
      // records ordered by kind (lines that miss the warp dropped), each
      // kind then runs its own class-free loop
      unsigned b[NKIND];
#pragma unroll
      for (int q = 0; q < NKIND; ++q) b[q] = __ballot_sync(0xffffffffu, r.kind == q + 1);
      const unsigned lt = (1u << lane) - 1u;
      int pos = 0, run = 0;
#pragma unroll
      for (int q = 0; q < NKIND; ++q) {
        if (r.kind == q + 1) pos = run + __popc(b[q] & lt);
        run += __popc(b[q]);
        nk[q] = run;
      }
      if (r.kind != KIND_MISS) {
        // per-point lines keep their chunk index (their GH3 constants are
        // formed from the record when needed)
        if (r.kind == KIND_REST && r.cls == CLS_MIXED) r.q1 = __int_as_float(j);
        wl[pos] = r;
      }
    }
    __syncwarp();
    span_lines<NSLOT, true, false>(wl, 0, nk[0], lanef, ngroup, sum, comp, part);
    span_lines<NSLOT, false, false>(wl, nk[0], nk[1], lanef, ngroup, sum, comp, part);
    span_lines<NSLOT, true, true>(wl, nk[1], nk[2], lanef, ngroup, sum, comp, part);
    span_lines<NSLOT, false, true>(wl, nk[2], nk[3], lanef, ngroup, sum, comp, part);
    if (COUNT) {
      cnt[2] += (unsigned long long)NSLOT * nk[1];
      cnt[1] += (unsigned long long)NSLOT * (nk[3] - nk[1]);
    }
    // the rest: GH1 or GH3 lines covering part of the span, and lines with a
    // method boundary, their core or their centre in the span
    for (int jj = nk[3]; jj < nk[4];) {
      const int je = min(nk[4], jj + KAHAN_GROUP - ngroup);
      ngroup += je - jj;
      for (; jj < je; ++jj) {
        const WarpLine &W = wl[jj];
        const int cls = W.cls;
        const int lo = W.lo, hi = W.hi;
        const float beta = W.beta, nphi = W.nphi, a2 = W.a2;
        // (i - c) of this lane's first point, exact in FP32
        const float d0 = W.d0 + lanef;
        if (cls == CLS_GH1) {
          const float P1 = W.q0;
#pragma unroll
          for (int k = 0; k < NSLOT; ++k) {
            const int i = wbase + lane + 32 * k;
            const float u = fmaf(d0 + (float)(32 * k), beta, nphi);
            const float r2 = fmaf(u, u, a2);
            const bool in = (unsigned)(i - lo) <= (unsigned)(hi - lo);
            part[k] += in ? P1 * fast_rcp(r2) : 0.0f;
            if (COUNT) cnt[2] += in;
          }
        } else if (cls == CLS_GH3) {
          const Gh3Line g3(a2, W.q0, W.q1, W.q2, W.q3);
#pragma unroll
          for (int k = 0; k < NSLOT; ++k) {
            const int i = wbase + lane + 32 * k;
            const float u = fmaf(d0 + (float)(32 * k), beta, nphi);
            const float r2 = fmaf(u, u, a2);
            const bool in = (unsigned)(i - lo) <= (unsigned)(hi - lo);
            part[k] = in ? g3.add(part[k], r2) : part[k];
            if (COUNT) cnt[1] += in;
          }
        } else {
          // Per point: GH1 or GH3; core points (r^2 < 100) are left to the
          // core kernel (k_core_f32).  Branch-free, so the slots stay
          // independent chains: the method's numerator and denominator are
          // selected before one reciprocal (the same operations, in the same
          // order, as the whole-span loops), and the sum is kept where the
          // point is outside the window or in the core.
          const int j = __float_as_int(W.q1);
          const float P1 = W.q0;
          const Gh3Line g3(a2, buf[j].P3);
#pragma unroll
          for (int k = 0; k < NSLOT; ++k) {
            const int i = wbase + lane + 32 * k;
            const float u = fmaf(d0 + (float)(32 * k), beta, nphi);
            const float r2 = fmaf(u, u, a2);
            float n, d;
            g3.nd(r2, n, d);  // not used (possibly infinite) where GH1 applies
            const bool gh1 = r2 >= 1.0e6f;
            const bool use = (unsigned)(i - lo) <= (unsigned)(hi - lo) && r2 >= 100.0f;
            const float t = fmaf(gh1 ? P1 : n, fast_rcp(gh1 ? r2 : d), part[k]);
            part[k] = use ? t : part[k];
            if (COUNT) {
              cnt[2] += use && gh1;
              cnt[1] += use && !gh1;
            }
          }
        }
      }
      if (ngroup == KAHAN_GROUP) kahan_fold<NSLOT>(ngroup, sum, comp, part);
    }
    __syncwarp();  // the group's records are overwritten next
    }
    // release the stage; the last warp out refills it
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&P.done[s], 1) == NW - 1) {
        P.done[s] = 0;
        __threadfence_block();
        f32_issue<LCH>(P, sl, seq + F32_STAGES, rec_all, nlines, tlo_all, thi_all, ntiles, cond_order, nitems,
                       st);
      }
    }
  }
}

// ------------------------------------------------- Algorithm 916 cores --
// The points of every line's core (fma(u, u, a^2) < 100 in the FP32
// arithmetic of k_voigt_f32, which skips exactly these points), one thread
// per grid point: the candidate lines of a warp's 32 points are those whose
// reference index lies within the condition's core reach of them (found by
// the warp's own search), screened by each line's core range from the pack;
// each thread adds S' K(|u|, a) of the lines whose core holds its point, in
// list order (deterministic), or appends the point to the surrogate's queue
// when routed.  The per-point sums go to kcore (every point written), so the
// kernel can run beside k_voigt_f32; k_core_add then adds them into kappa,
// rescaled like the main kernel's sums.  Few lines' cores overlap at a point
// (~4 at the medium workload), so the plain FP32 sum loses < 1e-7 relative.
constexpr int CORE_BLOCK = 128;

template <bool COUNT>
__global__ void __launch_bounds__(CORE_BLOCK)
    k_core_f32(const LineRec32 *__restrict__ rec_all, const int2 *__restrict__ core_all, int64_t nlines,
               const int32_t *__restrict__ ckey, int ngrid, float *__restrict__ kcore_all, CondStats *cst,
               SurrQueue *sq, const int *__restrict__ core_blk_all) {
  // per warp: the series weights of the line being evaluated
  __shared__ float s_w[CORE_BLOCK / 32][32];
  const int cond = blockIdx.y;
  const int cw1 = cst[cond].core_w1;
  if (cw1 == 0) return;  // no line of the condition has a core (k_core_add skips it too)
  // each warp finds its own 32 points' candidate lines: no CTA barrier
  const int64_t A = (int64_t)blockIdx.x * CORE_BLOCK + (threadIdx.x & ~31);
  if (A >= ngrid) return;  // warp-uniform
  const int lane = threadIdx.x & 31;
  float *w = s_w[threadIdx.x >> 5];
  const int64_t B = min(A + 32, (int64_t)ngrid);
  // The candidate window: the condition's largest core reach, or, when that
  // is below a block, the largest reach of the lines whose reference index
  // lies in this block or its two neighbours (no line from a farther block
  // reaches the warp); the core reach grows with the line centre, so the
  // low-wavenumber warps scan far fewer lines.
  int64_t W = cw1 - 1;
  if (W < CORE_BLK_PTS - 32) {
    const int nblk = core_blocks(ngrid);
    const int b = (int)(A / CORE_BLK_PTS);
    const int *cb = core_blk_all + (int64_t)cond * nblk;
    int r = cb[b];
    if (b > 0) r = max(r, cb[b - 1]);
    if (b + 1 < nblk) r = max(r, cb[b + 1]);
    W = r - 1;  // -1: no line near this block has a core
  }
  // integer searches (FP64 is the scarce unit here)
  const int64_t first = warp_search(ckey, 0, nlines, A - W, false);
  const int64_t last = warp_search(ckey, first, nlines, B - 1 + W, true);
  const LineRec32 *rec = rec_all + (int64_t)cond * nlines;
  const int2 *core = core_all + (int64_t)cond * nlines;
  const int i = (int)(A + lane);
  float v = 0.0f;
  unsigned long long n916 = 0, nterm = 0;
  // the line loop is warp-uniform: each line's weight table is built by the
  // whole warp when any lane's point lies in its core
  for (int64_t l = first; l < last; ++l) {
    const int2 cr = core[l];  // the line's core points, a superset of r^2 < 100
    bool in = i < ngrid && i >= cr.x && i <= cr.y;
    float u = 0.0f;
    const LineRec32 &L = rec[l];
    if (in) {
      u = fmaf((float)(i - L.c), L.beta, -L.phi_k);
      in = fmaf(u, u, L.a2) < 100.0f;
    }
    if (!__any_sync(0xffffffffu, in)) continue;
    w[lane] = a916_weight_f32(lane + 1, L.a2);
    __syncwarp();
    if (in) {
      v += core_point(L, fabsf(u), i, surr_row(sq, L.a), sq, cond, w);
      if (COUNT) {
        int n0, n1;
        a916_range_f32(fabsf(u), n0, n1);
        ++n916;
        nterm += (unsigned long long)(n1 - n0 + 1);
      }
    }
    __syncwarp();  // the table is rebuilt for the next line
  }
  if (i < ngrid) kcore_all[(int64_t)cond * ngrid + i] = v;
  if (COUNT) {
    for (int o = 16; o > 0; o >>= 1) {
      n916 += __shfl_down_sync(0xffffffffu, n916, o);
      nterm += __shfl_down_sync(0xffffffffu, nterm, o);
    }
    if (lane == 0 && n916) {
      atomicAdd(&cst[cond].region[0], n916);
      atomicAdd(&cst[cond].region[3], nterm);
    }
  }
}

// kappa += 2^E weight kcore at the points with a core sum (as k_voigt_f32's
// flush scales its sums); for weight 1 the scaled value is formed on the
// integer pipe, leaving one FP64 addition a point.
__global__ void __launch_bounds__(256)
    k_core_add(const float *__restrict__ kcore_all, int ngrid, double weight, double *__restrict__ kappa_all,
               const CondStats *cst) {
  const int cond = blockIdx.y;
  if (cst[cond].core_w1 == 0) return;
  const int E = cst[cond].scale_exp;
  const double scale = ldexp(weight, E);
  const bool unit = weight == 1.0;
  const float *kcore = kcore_all + (int64_t)cond * ngrid;
  double *kappa = kappa_all + (int64_t)cond * ngrid;
  // four points a thread per pass, their loads issued together
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < ngrid; i0 += 4 * stride) {
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q * stride;
      v[q] = i < ngrid ? kcore[i] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q * stride;
      if (v[q] != 0.0f) kappa[i] += unit ? scaled_to_double(v[q], E) : scale * (double)v[q];
    }
  }
}

cudaError_t launch_voigt_core(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o) {
  if (o.precision != HELK_PREC_F32_KAHAN || c->nlines <= 0) return cudaSuccess;
  SurrQueue *sq = o.surrogate ? c->squeue : nullptr;
  const dim3 grid((unsigned)((g.n + CORE_BLOCK - 1) / CORE_BLOCK), (unsigned)n_cond);
  ++c->launches;
  if (o.count_regions)
    k_core_f32<true><<<grid, CORE_BLOCK, 0, c->side_stream>>>(c->rec32, c->core_rng, c->nlines, c->ckey32,
                                                               (int)g.n, c->kcore, c->cstats, sq, c->core_blk);
  else
    k_core_f32<false><<<grid, CORE_BLOCK, 0, c->side_stream>>>(c->rec32, c->core_rng, c->nlines, c->ckey32,
                                                                (int)g.n, c->kcore, c->cstats, sq, c->core_blk);
  return cudaGetLastError();
}

cudaError_t launch_core_add(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o, double *kappa) {
  if (o.precision != HELK_PREC_F32_KAHAN || c->nlines <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<int64_t>((g.n + 255) / 256, (int64_t)c->num_sms * 8), (unsigned)n_cond);
  ++c->launches;
  k_core_add<<<grid, 256, 0, c->stream>>>(c->kcore, (int)g.n, o.weight, kappa, c->cstats);
  return cudaGetLastError();
}

// --------------------------------------------------------------- launch --
// FP32 kernel shapes, X(warps per CTA, slots per warp, candidate lines per
// pipeline stage, resident CTAs per SM the kernel is compiled for); a shape's
// code is its 1-based position in the list.  NSLOT is a template parameter
// (no per-slot bounds test in the hot loops) and the tile is 32 warps NSLOT
// points.  With 8 warps and 128-line stages the slots span 6..16, so that
// the number of tiles can be matched to whole waves of resident CTAs (equal
// tiles finish together, so a partial last wave idles the rest of the GPU);
// the other entries vary the CTA size (4, 12 warps) and the stage length (64,
// 256 lines, the latter also with 10-12 slots) for the autotuner.
#define HELK_F32_SHAPES(X)                                                                          \
  X(8, 6, 128, 3) X(8, 7, 128, 3) X(8, 8, 128, 3) X(8, 9, 128, 2) X(8, 10, 128, 2) X(8, 11, 128, 2)   \
  X(8, 12, 128, 2) X(8, 13, 128, 2) X(8, 14, 128, 2) X(8, 16, 128, 2) X(8, 8, 64, 3) X(8, 8, 256, 3)  \
  X(8, 7, 256, 3) X(4, 8, 128, 6) X(4, 9, 128, 4) X(12, 8, 128, 2) X(8, 10, 256, 2) X(8, 11, 256, 2)  \
  X(8, 12, 256, 2)
constexpr int F32_COUNT_CODE = 3;  // the counting variant (statistics): 8 warps, 8 slots, 128 lines
constexpr int F32_COUNT_NSLOT = 8, F32_COUNT_WARPS = 8, F32_COUNT_LCH = 128;

struct F32Shape {
  int warps, nslot, lch;
};
static const F32Shape kF32Shapes[] = {
#define X(W, NS, L, MB) {W, NS, L},
    HELK_F32_SHAPES(X)
#undef X
};
constexpr int F32_NSHAPES = (int)(sizeof(kF32Shapes) / sizeof(kF32Shapes[0]));

template <int W, int NS, int L, int MB>
static int f32_slots(helk_ctx *c) {
  return resident_ctas(c, k_voigt_f32<32 * W, NS, L, false, MB>, 32 * W);
}

bool voigt_shape_info(int precision, int code, int *points, int *warps, int *lines_per_stage) {
  if (precision != HELK_PREC_F32_KAHAN) return f64_shape_info(code, points, warps, lines_per_stage);
  if (code < 1 || code > F32_NSHAPES) return false;
  const F32Shape &s = kF32Shapes[code - 1];
  if (points) *points = 32 * s.warps * s.nslot;
  if (warps) *warps = s.warps;
  if (lines_per_stage) *lines_per_stage = s.lch;
  return true;
}

int voigt_shape_candidates(int precision, int *out, int max) {
  if (precision != HELK_PREC_F32_KAHAN) return f64_shape_candidates(out, max);
  int n = 0;
  for (int code = 1; code <= F32_NSHAPES && n < max; ++code) out[n++] = code;
  return n;
}

// Wave efficiency of ceil(n / tile) equal tiles on `slots` resident CTAs,
// times the share of a (line, warp) pair's work that is evaluation (the
// pair's fixed cost is about 2.5 slots).
static double f32_tile_score(int64_t n, int tile, int p, int slots) {
  const int64_t ntiles = (n + tile - 1) / tile;
  const double waves = (double)ntiles / slots;
  return waves / ceil(waves) * p / (p + 2.5);
}

int voigt_shape(helk_ctx *c, int precision, int count, int64_t n) {
  const int prec = precision == HELK_PREC_F32_KAHAN ? 1 : 0;
  if (!count && c->tuned_tile[prec] > 0 && c->tuned_n[prec] == n) return c->tuned_tile[prec];
  if (precision != HELK_PREC_F32_KAHAN) return f64_shape(c, count, n);
  if (count) return F32_COUNT_CODE;
  // without timing: the 8-warp, 128-line shapes by wave efficiency
  int best = F32_COUNT_CODE, code = 0;
  double best_score = -1.0;
#define X(W, NS, L, MB)                                                                  \
  ++code;                                                                                \
  if (W == 8 && L == 128) {                                                              \
    const double sc = f32_tile_score(n, 32 * W * NS, NS, f32_slots<W, NS, L, MB>(c));    \
    if (sc > best_score + 1e-9) {                                                        \
      best_score = sc;                                                                   \
      best = code;                                                                       \
    }                                                                                    \
  }
  HELK_F32_SHAPES(X)
#undef X
  return best;
}

cudaError_t launch_voigt(helk_ctx *c, int n_cond, const helk_grid &g, const helk_opts &o,
                         double *kappa, int shape, int64_t ntiles) {
  const int64_t nitems = ntiles * n_cond;
  if (o.precision != HELK_PREC_F32_KAHAN) return launch_voigt_f64(c, n_cond, g, o, kappa, shape, ntiles);
  SurrQueue *sq = o.surrogate ? c->squeue : nullptr;
  if (o.count_regions) {
    if (shape != F32_COUNT_CODE) return cudaErrorInvalidValue;
    constexpr int B = 32 * F32_COUNT_WARPS;
    auto kern = k_voigt_f32<B, F32_COUNT_NSLOT, F32_COUNT_LCH, true, 3>;
    ++c->launches;
    kern<<<persistent_grid(c, kern, B, nitems), B, 0, c->stream>>>(
        c->rec32, c->nlines, c->tile_lo, c->tile_hi, ntiles, c->cond_order, n_cond, (int)g.n, o.weight,
        o.accumulate, kappa, c->cstats, c->stats, sq);
    return cudaGetLastError();
  }
  int code = 0;
#define X(W, NS, L, MB)                                                                           \
  if (++code == shape) {                                                                          \
    auto kern = k_voigt_f32<32 * W, NS, L, false, MB>;                                             \
    ++c->launches;                                                                                 \
    kern<<<persistent_grid(c, kern, 32 * W, nitems), 32 * W, 0, c->stream>>>(                      \
        c->rec32, c->nlines, c->tile_lo, c->tile_hi, ntiles, c->cond_order, n_cond, (int)g.n,      \
        o.weight, o.accumulate, kappa, c->cstats, c->stats, sq);                                   \
    return cudaGetLastError();                                                                    \
  }
  HELK_F32_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace helk
