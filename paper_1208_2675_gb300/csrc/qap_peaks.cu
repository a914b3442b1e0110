// qap_peaks.cu -- microbenchmarks of the figures that bound the SA kernels
// (include/qap_peaks.h): shared-memory and L2 bandwidth, 32-bit integer and
// dp4a issue rates, and the latencies of a CTA barrier, a cluster barrier, a
// grid barrier and of dependent loads from shared memory, a peer CTA's shared
// memory and L2.  Each kernel is short and in bounds by construction; the one
// spin-wait (the grid barrier) is bounded and reports a timeout.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "qap_peaks.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kSmemInts4 = 4096;      // 64 KB of int4 in the bandwidth kernel
constexpr int kChainWords = 8192;     // 32 KB chain in the latency kernels
constexpr unsigned kGridSpinLimit = 1u << 21;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ld.shared.v4 streaming: every thread reads four fixed 16-byte slots, one per
// quarter of the buffer, consecutive across a warp (no bank conflicts); the
// loads are volatile so that none of the repeated loads is optimised away.
__global__ void __launch_bounds__(1024) pk_smem_bw(int iters, unsigned long long *cycles,
                                                   unsigned *sink) {
  extern __shared__ int4 buf[];
  const int t = threadIdx.x;
  for (int i = t; i < kSmemInts4; i += blockDim.x) buf[i] = make_int4(i, i + 1, i + 2, i + 3);
  __syncthreads();
  const unsigned base = smem_addr(buf);
  unsigned a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = base + 16u * (unsigned)((t + q * 1024) & (kSmemInts4 - 1));
  unsigned acc = 0;
  const long long c0 = clock64();
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned x, y, z, w;
      asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a[q]));
      acc ^= x ^ y ^ z ^ w;
    }
  }
  __syncthreads();
  const long long c1 = clock64();
  if (t == 0) cycles[blockIdx.x] = (unsigned long long)(c1 - c0);
  if (acc == 0x9E3779B9u) sink[0] = acc;
}

// ld.global.cg (L2, not L1) of an L2-resident buffer, grid-stride, four loads
// in flight per thread.
__global__ void pk_l2_bw(const int4 *buf, long long n4, int passes, unsigned *sink) {
  unsigned acc = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      const int4 v0 = __ldcg(buf + i), v1 = __ldcg(buf + i + stride);
      const int4 v2 = __ldcg(buf + i + 2 * stride), v3 = __ldcg(buf + i + 3 * stride);
      acc ^= v0.x ^ v0.y ^ v0.z ^ v0.w ^ v1.x ^ v1.y ^ v1.z ^ v1.w;
      acc ^= v2.x ^ v2.y ^ v2.z ^ v2.w ^ v3.x ^ v3.y ^ v3.z ^ v3.w;
    }
    for (; i < n4; i += stride) {
      const int4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  if (acc == 0x9E3779B9u) sink[0] = acc;
}

__global__ void pk_fill(int4 *buf, long long n4) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x)
    buf[i] = make_int4((int)i, (int)(i >> 7), 1, 2);
}

// Eight independent chains of 32-bit multiply-adds per thread.
__global__ void __launch_bounds__(1024) pk_imad(int iters, unsigned seed,
                                                unsigned long long *cycles, unsigned *sink) {
  unsigned x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 8u + j + seed;
  const unsigned m = seed | 1u, c = seed >> 3;
  __syncthreads();
  const long long c0 = clock64();
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(m), "r"(c));
  }
  __syncthreads();
  const long long c1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(c1 - c0);
  unsigned acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc ^= x[j];
  if (acc == 0x9E3779B9u) sink[0] = acc;
}

// Eight independent chains of dp4a per thread.
__global__ void __launch_bounds__(1024) pk_dp4a(int iters, unsigned seed,
                                                unsigned long long *cycles, unsigned *sink) {
  int x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (int)(threadIdx.x * 8u + j + seed);
  const int a = (int)(seed * 0x01010101u), b = (int)(seed ^ 0x7F3F1F0Fu);
  __syncthreads();
  const long long c0 = clock64();
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        asm volatile("dp4a.s32.s32 %0, %1, %2, %0;" : "+r"(x[j]) : "r"(a), "r"(b));
  }
  __syncthreads();
  const long long c1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(c1 - c0);
  int acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc ^= x[j];
  if (acc == 0x1E3779B9) sink[0] = (unsigned)acc;
}

__global__ void __launch_bounds__(640) pk_cta_barrier(int iters, unsigned long long *cycles) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const long long c0 = clock64();
  for (int k = 0; k < iters; ++k) {
    if (threadIdx.x == (unsigned)(k & 511)) s += k;
    __syncthreads();
  }
  const long long c1 = clock64();
  if (threadIdx.x == 0) cycles[0] = (unsigned long long)(c1 - c0) + (s == -1 ? 1 : 0);
}

__global__ void pk_cluster_barrier(int iters, unsigned long long *cycles) {
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const long long c0 = clock64();
  for (int k = 0; k < iters; ++k) cl.sync();
  const long long c1 = clock64();
  if (cl.block_rank() == 0 && threadIdx.x == 0) cycles[0] = (unsigned long long)(c1 - c0);
}

// A grid barrier as a persistent single-chain kernel would build it: every CTA
// adds 1 to a monotonic counter with release semantics and waits (acquire)
// until it reaches (k + 1) * gridDim.x.  The wait gives up after a bounded
// number of polls and flags an error.
__global__ void pk_grid_barrier(int iters, unsigned *counter, int *err,
                                unsigned long long *cycles) {
  __shared__ int s_abort;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  const unsigned G = gridDim.x;
  const long long c0 = clock64();
  int k = 0;
  for (; k < iters; ++k) {
    if (threadIdx.x == 0) {
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
      const unsigned target = (unsigned)(k + 1) * G;
      unsigned v = 0, polls = 0;
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
        if ((int)(v - target) >= 0) break;
        if (++polls > kGridSpinLimit) {
          atomicExch(err, 1);
          s_abort = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (s_abort) break;
  }
  const long long c1 = clock64();
  if (blockIdx.x == 0 && threadIdx.x == 0) cycles[0] = (unsigned long long)(c1 - c0);
}

__global__ void pk_chain_init(unsigned *chain, unsigned n, unsigned step) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    chain[i] = (i + step) % n;
}

// One thread follows idx = chain[idx] with ld.global.cg; a first pass brings
// the visited lines into L2, the second is timed.
__global__ void pk_l2_latency(const unsigned *chain, int hops, unsigned long long *cycles,
                              unsigned *sink) {
  unsigned idx = 0;
  for (int k = 0; k < hops; ++k) idx = __ldcg(chain + idx);
  idx = 0;
  const long long c0 = clock64();
  for (int k = 0; k < hops; ++k) idx = __ldcg(chain + idx);
  const long long c1 = clock64();
  cycles[0] = (unsigned long long)(c1 - c0);
  sink[0] = idx;
}

// Rank 1 of a 2-CTA cluster holds a chain in its shared memory; thread 0 of
// rank 0 follows it through ld.shared::cluster, then through its own copy with
// ld.shared.
__global__ void pk_dsmem_latency(int hops, unsigned long long *cycles, unsigned *sink) {
  __shared__ unsigned chain[kChainWords];
  cg::cluster_group cl = cg::this_cluster();
  for (int i = threadIdx.x; i < kChainWords; i += blockDim.x)
    chain[i] = (unsigned)((i + 33 * 32 + 1) % kChainWords);
  cl.sync();
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    unsigned remote = 0;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 1;" : "=r"(remote) : "r"(smem_addr(chain)));
    unsigned idx = 0;
    const long long c0 = clock64();
    for (int k = 0; k < hops; ++k)
      asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(idx) : "r"(remote + 4u * idx));
    const long long c1 = clock64();
    const unsigned local = smem_addr(chain);
    unsigned j = 0;
    const long long c2 = clock64();
    for (int k = 0; k < hops; ++k)
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(j) : "r"(local + 4u * j));
    const long long c3 = clock64();
    cycles[0] = (unsigned long long)(c1 - c0);
    cycles[1] = (unsigned long long)(c3 - c2);
    sink[0] = idx ^ j;
  }
  cl.sync();  // rank 1 keeps its shared memory until rank 0 is done
}

struct Scratch {
  unsigned long long *cyc = nullptr;  // per-block cycle counts (device)
  unsigned *sink = nullptr;
  int *err = nullptr;
  unsigned *counter = nullptr;
  int4 *buf = nullptr;
  ~Scratch() {
    cudaFree(cyc);
    cudaFree(sink);
    cudaFree(err);
    cudaFree(counter);
    cudaFree(buf);
  }
};

#define PK_CK(call)                                              \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess)                                       \
      return e_ == cudaErrorMemoryAllocation ? QAP_E_NOMEM : QAP_E_CUDA; \
  } while (0)

// Median-free: the mean of the per-block cycle counts.
double mean_cycles(const unsigned long long *h, int n) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += (double)h[i];
  return n ? s / n : 0.0;
}

}  // namespace

extern "C" int qap_peaks_measure(qap_peaks *out) {
  if (!out) return QAP_E_INVAL;
  memset(out, 0, sizeof *out);
  int dev = 0, sms = 0, optin = 0, l2 = 0;
  PK_CK(cudaGetDevice(&dev));
  PK_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PK_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PK_CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
  out->sm_count = sms;
  out->smem_optin_bytes = optin;
  out->l2_bytes = l2;
  if (sms < 1 || sms > 4096) return QAP_E_CUDA;

  Scratch s;
  const long long n4 = (32ll << 20) / 16;  // 32 MB
  PK_CK(cudaMalloc(&s.cyc, sizeof(unsigned long long) * 4096));
  PK_CK(cudaMalloc(&s.sink, sizeof(unsigned) * 4));
  PK_CK(cudaMalloc(&s.err, sizeof(int)));
  PK_CK(cudaMalloc(&s.counter, sizeof(unsigned)));
  PK_CK(cudaMalloc(&s.buf, (size_t)n4 * 16 * 2));  // 64 MB: the L2 buffer, then the chain
  cudaEvent_t e0, e1;
  PK_CK(cudaEventCreate(&e0));
  PK_CK(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } evg{e0, e1};
  unsigned long long hc[4096];
  float ms = 0.f;

  // ---- shared-memory bandwidth and the SM clock ----
  {
    const int iters = 20000, smem = kSmemInts4 * 16;
    PK_CK(cudaFuncSetAttribute(pk_smem_bw, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    pk_smem_bw<<<sms, 1024, smem>>>(iters / 10, s.cyc, s.sink);  // warm-up
    PK_CK(cudaEventRecord(e0));
    pk_smem_bw<<<sms, 1024, smem>>>(iters, s.cyc, s.sink);
    PK_CK(cudaEventRecord(e1));
    PK_CK(cudaEventSynchronize(e1));
    PK_CK(cudaGetLastError());
    PK_CK(cudaEventElapsedTime(&ms, e0, e1));
    PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost));
    const double cyc = mean_cycles(hc, sms);
    const double bytes_cta = 1024.0 * 16.0 * 4.0 * iters;
    out->smem_bytes_per_clk_sm = cyc > 0 ? bytes_cta / cyc : 0.0;
    out->sm_mhz = ms > 0 ? cyc / (ms * 1e3) : 0.0;
    out->smem_gbs_chip = ms > 0 ? bytes_cta * sms / (ms * 1e-3) / 1e9 : 0.0;
  }
  const double mhz = out->sm_mhz > 0 ? out->sm_mhz : 1.0;

  // ---- L2 bandwidth (32 MB buffer, read 40 times) ----
  {
    pk_fill<<<4 * sms, 256>>>(s.buf, n4);
    pk_l2_bw<<<4 * sms, 512>>>(s.buf, n4, 2, s.sink);  // bring it into L2
    const int passes = 40;
    PK_CK(cudaEventRecord(e0));
    pk_l2_bw<<<4 * sms, 512>>>(s.buf, n4, passes, s.sink);
    PK_CK(cudaEventRecord(e1));
    PK_CK(cudaEventSynchronize(e1));
    PK_CK(cudaGetLastError());
    PK_CK(cudaEventElapsedTime(&ms, e0, e1));
    out->l2_gbs = ms > 0 ? (double)n4 * 16.0 * passes / (ms * 1e-3) / 1e9 : 0.0;
    // one SM: the first 8 MB of the (L2-resident) buffer, read by one CTA
    const long long m4 = n4 < (1ll << 19) ? n4 : (1ll << 19);
    const int passes1 = 4;
    PK_CK(cudaEventRecord(e0));
    pk_l2_bw<<<1, 1024>>>(s.buf, m4, passes1, s.sink);
    PK_CK(cudaEventRecord(e1));
    PK_CK(cudaEventSynchronize(e1));
    PK_CK(cudaGetLastError());
    PK_CK(cudaEventElapsedTime(&ms, e0, e1));
    out->l2_gbs_sm = ms > 0 ? (double)m4 * 16.0 * passes1 / (ms * 1e-3) / 1e9 : 0.0;
  }

  // ---- integer issue rates ----
  {
    const int iters = 4000;
    pk_imad<<<sms, 1024>>>(iters / 10, 12345u, s.cyc, s.sink);
    pk_imad<<<sms, 1024>>>(iters, 12345u, s.cyc, s.sink);
    PK_CK(cudaDeviceSynchronize());
    PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost));
    double cyc = mean_cycles(hc, sms);
    out->int32_ops_per_clk_sm = cyc > 0 ? 1024.0 * 64.0 * iters / cyc : 0.0;
    pk_dp4a<<<sms, 1024>>>(iters / 10, 12345u, s.cyc, s.sink);
    pk_dp4a<<<sms, 1024>>>(iters, 12345u, s.cyc, s.sink);
    PK_CK(cudaDeviceSynchronize());
    PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost));
    cyc = mean_cycles(hc, sms);
    out->dp4a_per_clk_sm = cyc > 0 ? 1024.0 * 64.0 * iters / cyc : 0.0;
  }

  // ---- CTA barrier, 640 threads ----
  {
    const int iters = 20000;
    pk_cta_barrier<<<1, 640>>>(iters, s.cyc);
    PK_CK(cudaDeviceSynchronize());
    PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    out->cta_barrier_ns = (double)hc[0] / iters / mhz * 1e3;
  }

  // ---- cluster barriers ----
  {
    cudaFuncSetAttribute(pk_cluster_barrier, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    const int sizes[5] = {2, 4, 8, 13, 16};
    const int iters = 20000;
    for (int k = 0; k < 5; ++k) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = sizes[k];
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(sizes[k]);
      cfg.blockDim = dim3(128);
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, pk_cluster_barrier, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        continue;
      }
      if (cudaLaunchKernelEx(&cfg, pk_cluster_barrier, iters, s.cyc) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      PK_CK(cudaDeviceSynchronize());
      PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
      out->cluster_barrier_ns[k] = (double)hc[0] / iters / mhz * 1e3;
    }
  }

  // ---- grid barrier, one CTA per SM, cooperative launch ----
  {
    int iters = 4000;
    PK_CK(cudaMemset(s.counter, 0, sizeof(unsigned)));
    PK_CK(cudaMemset(s.err, 0, sizeof(int)));
    void *args[] = {&iters, &s.counter, &s.err, &s.cyc};
    PK_CK(cudaLaunchCooperativeKernel((const void *)pk_grid_barrier, dim3(sms), dim3(128), args,
                                      0, 0));
    PK_CK(cudaDeviceSynchronize());
    int herr = 0;
    PK_CK(cudaMemcpy(&herr, s.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return QAP_E_TIMEOUT;
    PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    out->grid_barrier_ns = (double)hc[0] / iters / mhz * 1e3;
  }

  // ---- dependent-load latencies ----
  {
    unsigned *chain = reinterpret_cast<unsigned *>(s.buf + n4);  // second 32 MB
    const unsigned n = (unsigned)((32ll << 20) / 4);
    pk_chain_init<<<4 * sms, 256>>>(chain, n, 32u * 997u + 7u);
    const int hops = 20000;
    pk_l2_latency<<<1, 1>>>(chain, hops, s.cyc, s.sink);
    PK_CK(cudaDeviceSynchronize());
    PK_CK(cudaMemcpy(hc, s.cyc, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    out->l2_latency_ns = (double)hc[0] / hops / mhz * 1e3;

    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(128);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, pk_dsmem_latency, hops, s.cyc, s.sink) == cudaSuccess) {
      PK_CK(cudaDeviceSynchronize());
      PK_CK(cudaMemcpy(hc, s.cyc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
      out->dsmem_latency_ns = (double)hc[0] / hops / mhz * 1e3;
      out->smem_latency_ns = (double)hc[1] / hops / mhz * 1e3;
    } else {
      cudaGetLastError();
    }
  }
  PK_CK(cudaGetLastError());
  return QAP_OK;
}
