// roofline_probe.cu -- microbenchmarks of the memory roofs that bound the
// propagation kernels: shared-memory loads (16-byte, conflict-free), the
// relaxed shared atomics that carry the tells, 8-byte interval loads at
// scattered indices (the kernels' gather pattern) and L2 reads.  Every loop
// is bounded by its iteration count; no kernel waits on another.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pccp.h"
#include "../../include/pccp_probe.h"

namespace {

// One 1024-thread CTA per SM (32 warps: enough to saturate shared memory and,
// with four loads in flight per thread, L2), so the first CTA's clock64 span
// is the launch's span in SM cycles.
constexpr int kThreads = 1024;
constexpr int kCtasPerSm = 1;
constexpr int kSmemWords = 8192;  // 32 KB per CTA

__device__ __forceinline__ uint32_t sa(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void stamp(long long* cyc, long long t0) {
  if (blockIdx.x == 0 && threadIdx.x == 0) cyc[0] = clock64() - t0;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    k_smem_load(int iters, uint32_t* sink, long long* cyc) {
  __shared__ __align__(16) uint32_t buf[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) buf[i] = i * 2654435761u;
  __syncthreads();
  const long long t0 = clock64();
  uint32_t acc = 0;
  // a warp reads 32 consecutive 16-byte words: every bank once per wavefront
  int idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int q = (idx + 128 * k) & (kSmemWords / 4 - 1);
      uint32_t a, b, c, d;
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                   : "r"(sa(buf + 4 * q)));
      acc ^= a ^ b ^ c ^ d;
    }
    idx += 32;
  }
  __syncthreads();
  stamp(cyc, t0);
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    k_smem_atom(int iters, uint32_t* sink, long long* cyc) {
  __shared__ __align__(16) int buf[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) buf[i] = 0;
  __syncthreads();
  const long long t0 = clock64();
  int acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // lane l of every warp hits bank l: conflict-free
      const int w = (threadIdx.x + kThreads * k) & (kSmemWords - 1);
      int old;
      asm volatile("atom.relaxed.cta.shared::cta.max.s32 %0, [%1], %2;"
                   : "=r"(old)
                   : "r"(sa(buf + w)), "r"(it + k)
                   : "memory");
      acc ^= old;
    }
  }
  __syncthreads();
  stamp(cyc, t0);
  if (acc == 0x1234567) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    k_smem_dom(int iters, uint32_t* sink, long long* cyc) {
  __shared__ __align__(16) int2 buf[kSmemWords / 2];
  for (int i = threadIdx.x; i < kSmemWords / 2; i += blockDim.x) buf[i] = make_int2(i, i + 1);
  __syncthreads();
  const long long t0 = clock64();
  // a pseudo-random start per thread (top bits of a multiplicative hash):
  // lanes gather from random banks
  int p = static_cast<int>(((threadIdx.x + 1024u * blockIdx.x) * 2654435761u) >> 20) &
          (kSmemWords / 2 - 1);
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int q = (p + 613 * k) & (kSmemWords / 2 - 1);
      int a, b;
      asm volatile("ld.relaxed.cta.shared::cta.v2.s32 {%0, %1}, [%2];"
                   : "=r"(a), "=r"(b)
                   : "r"(sa(buf + q)));
      acc ^= static_cast<uint32_t>(a + b);
    }
    p = (p + 8 * 613 + 1) & (kSmemWords / 2 - 1);
  }
  __syncthreads();
  stamp(cyc, t0);
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    k_l2_read(const uint4* __restrict__ src, long long n16, int iters, uint32_t* sink,
              long long* cyc) {
  const long long t0 = clock64();
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
    long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {  // four loads in flight
      uint32_t r[16];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r[4 * u]), "=r"(r[4 * u + 1]), "=r"(r[4 * u + 2]), "=r"(r[4 * u + 3])
                     : "l"(src + i + u * stride));
#pragma unroll
      for (int u = 0; u < 16; ++u) acc ^= r[u];
    }
    for (; i < n16; i += stride) {
      uint32_t a, b, c, d;
      asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                   : "l"(src + i));
      acc ^= a ^ b ^ c ^ d;
    }
  }
  __syncthreads();
  stamp(cyc, t0);
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

constexpr long long kL2Bytes = 32ll << 20;

}  // namespace

extern "C" int pccp_probe(int kind, int iters, pccp_probe_result* out) {
  if (!out || kind < PCCP_PROBE_SMEM_LOAD || kind > PCCP_PROBE_L2_READ) return PCCP_ERR_INVALID;
  int dev = 0, n_sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PCCP_ERR_CUDA;
  if (iters <= 0) {
    const int dflt[4] = {40000, 64000, 40000, 6000};
    iters = dflt[kind];
  }
  const int ctas = n_sms * kCtasPerSm;
  uint32_t* sink = nullptr;
  long long* cyc = nullptr;
  uint4* l2 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PCCP_OK;
  float ms = 0.f;
  long long cycles = 0;
  const long long n16 = kL2Bytes / 16;
  auto launch = [&](int n_iters) {
    switch (kind) {
      case PCCP_PROBE_SMEM_LOAD: k_smem_load<<<ctas, kThreads>>>(n_iters, sink, cyc); break;
      case PCCP_PROBE_SMEM_ATOM: k_smem_atom<<<ctas, kThreads>>>(n_iters, sink, cyc); break;
      case PCCP_PROBE_SMEM_DOM: k_smem_dom<<<ctas, kThreads>>>(n_iters, sink, cyc); break;
      default: k_l2_read<<<ctas, kThreads>>>(l2, n16, n_iters, sink, cyc); break;
    }
    return cudaGetLastError();
  };
  if (cudaMalloc(&sink, sizeof(uint32_t) * ctas) != cudaSuccess ||
      cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess ||
      (kind == PCCP_PROBE_L2_READ && cudaMalloc(&l2, kL2Bytes) != cudaSuccess) ||
      (l2 && cudaMemset(l2, 1, kL2Bytes) != cudaSuccess) ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = PCCP_ERR_CUDA;
  } else if (launch(iters > 4 ? iters / 4 : 1) != cudaSuccess ||  // warm-up
             cudaEventRecord(e0) != cudaSuccess || launch(iters) != cudaSuccess ||
             cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
             cudaMemcpy(&cycles, cyc, sizeof(cycles), cudaMemcpyDeviceToHost) != cudaSuccess) {
    rc = PCCP_ERR_CUDA;
  }
  if (rc == PCCP_OK) {
    const double threads = static_cast<double>(ctas) * kThreads;
    double work = 0.0;
    switch (kind) {
      case PCCP_PROBE_SMEM_LOAD: work = threads * iters * 8.0 * 16.0; break;
      case PCCP_PROBE_SMEM_ATOM: work = threads * iters * 8.0; break;
      case PCCP_PROBE_SMEM_DOM: work = threads * iters * 8.0 * 8.0; break;
      default: work = static_cast<double>(kL2Bytes) * iters; break;
    }
    out->work = work;
    out->ms = ms;
    out->sm_cycles = static_cast<double>(cycles);
    out->n_sms = n_sms;
    out->ctas = ctas;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (l2) cudaFree(l2);
  if (cyc) cudaFree(cyc);
  if (sink) cudaFree(sink);
  return rc;
}
