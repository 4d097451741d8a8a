// k_probe.cu -- throughput probes of the arithmetic units that bound the
// Voigt kernels: FP32 FMA (the FP32 form's pipe), FP64 FMA (the FP64 form's
// pipe) and the MUFU reciprocal and base-2 exponential (the co-bound of the
// FP32 form and of the surrogate's activations).  Each probe fills every SM
// with independent dependency chains of one instruction and is timed with
// CUDA events on the context stream, so the roofline fractions the benchmark
// reports are taken against rates measured on the GPU at hand, at the clock
// it runs at, rather than against unit counts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "helk_internal.cuh"

namespace helk {

constexpr int PR_THREADS = 512;
constexpr int PR_CHAINS = 8;   // independent chains per thread
constexpr int PR_UNROLL = 16;  // instructions per chain per loop iteration

__device__ __forceinline__ float mufu_rcp(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float mufu_ex2(float x) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// KIND: HELK_PROBE_*.  The chains' values stay bounded (x -> a x + b with
// |a| < 1; x -> 1/(x + b); x -> 2^-|x| in (0, 1]); the final store is
// conditional on a value the chains never reach, so the work cannot be
// removed.  The reciprocal probe issues one FP32 addition per reciprocal,
// which costs issue slots but not MUFU throughput.
template <int KIND>
__global__ void __launch_bounds__(PR_THREADS) k_probe(int iters, float a, float b, double ad, double bd,
                                                      float *sink_f, double *sink_d) {
  const float seed = 1.0f + 1.0e-3f * (float)(threadIdx.x & 63);
  if (KIND == HELK_PROBE_DFMA) {
    double x[PR_CHAINS];
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = (double)seed + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < PR_UNROLL; ++u)
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) x[c] = fma(x[c], ad, bd);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
    if (s == -1.0) sink_d[blockIdx.x] = s;
  } else {
    float x[PR_CHAINS];
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = seed + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < PR_UNROLL; ++u)
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) {
          if (KIND == HELK_PROBE_FFMA) x[c] = fmaf(x[c], a, b);
          // x -> 1/(x + b): an addition between the reciprocals, since the
          // compiler may fold two reciprocals in a row into nothing
          if (KIND == HELK_PROBE_MUFU_RCP) x[c] = mufu_rcp(x[c] + b);
          if (KIND == HELK_PROBE_MUFU_EX2) x[c] = mufu_ex2(-fabsf(x[c]));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
    if (s == -1.0f) sink_f[blockIdx.x] = s;
  }
}

template <int KIND>
static cudaError_t run_probe(helk_ctx *c, int iters, int blocks, float *sink_f, double *sink_d) {
  ++c->launches;
  k_probe<KIND><<<blocks, PR_THREADS, 0, c->stream>>>(iters, 0.999999f, 1.0e-6f, 0.999999, 1.0e-6, sink_f,
                                                      sink_d);
  return cudaGetLastError();
}

cudaError_t launch_probe(helk_ctx *c, int kind, int iters, int blocks, void *sink) {
  float *sf = static_cast<float *>(sink);
  double *sd = static_cast<double *>(sink);
  switch (kind) {
    case HELK_PROBE_FFMA: return run_probe<HELK_PROBE_FFMA>(c, iters, blocks, sf, sd);
    case HELK_PROBE_DFMA: return run_probe<HELK_PROBE_DFMA>(c, iters, blocks, sf, sd);
    case HELK_PROBE_MUFU_RCP: return run_probe<HELK_PROBE_MUFU_RCP>(c, iters, blocks, sf, sd);
    case HELK_PROBE_MUFU_EX2: return run_probe<HELK_PROBE_MUFU_EX2>(c, iters, blocks, sf, sd);
    default: return cudaErrorInvalidValue;
  }
}

int probe_blocks(helk_ctx *c) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_probe<HELK_PROBE_FFMA>, PR_THREADS, 0) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return occ * c->num_sms;
}

// Instructions of the probed kind per thread per loop iteration.
int probe_ops_per_iter() { return PR_CHAINS * PR_UNROLL; }
int probe_threads() { return PR_THREADS; }

}  // namespace helk
