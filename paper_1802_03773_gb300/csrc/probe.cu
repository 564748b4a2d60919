// Peak-rate probes of this GPU for the roofline denominators that no library measures: FP32
// and FP64 fused multiply-add throughput of the CUDA cores, and the dense TF32 rate of the
// 5th-generation tensor cores (tcgen05.mma kind::tf32, M = 128, N = 256, K = 8 per
// instruction, FP32 accumulation in tensor memory).  Each probe is one launch over every SM,
// timed with CUDA events; the rates are returned in TFLOP/s (2 flops per multiply-add).  The
// host-link probe times the two ways inputs in host memory reach a kernel: a copy-engine copy
// into device memory, and a kernel reading pinned host memory directly.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "internal.h"

namespace qrkit {
namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kFmaThreads = 256;
constexpr int kTcThreads = 128;
constexpr int kTcN = 256;           // MMA N (tensor memory columns of the accumulator)
constexpr uint32_t kTcWait = 1u << 26;

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_probe_kernel(T seed, int iters, T* sink) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
  const T m = (T)0.999999, k = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (T)-1) sink[0] = s;   // never true: keeps the chains alive
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no-swizzle operand descriptor (8-row x 16-byte core matrices, LBO 128 B, SBO 1024 B)
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// One CTA per SM: A (128 x 8 tf32) and B (256 x 8 tf32) zero in shared memory, `iters` MMAs
// into one tensor-memory accumulator, issued by one thread, then one commit and a bounded wait.
// The operands use the layout of the descriptors above: an 8-row group every 1024 bytes, of
// which the two 128-byte core matrices of K = 8 are read.
constexpr int kTcSmem = (128 / 8 + kTcN / 8) * 1024;
__global__ void __launch_bounds__(kTcThreads, 1) tf32_probe_kernel(int iters, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;                     // 16 row groups
  unsigned char* B = smem + (128 / 8) * 1024;  // 32 row groups
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mbar;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < kTcSmem / 4; e += kTcThreads) reinterpret_cast<uint32_t*>(smem)[e] = 0u;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    // D f32, A and B tf32, K-major; N >> 3 at bits 17-22, M >> 4 at bits 24-28
    const uint32_t id = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint64_t ad = desc(su32(A)), bd = desc(su32(B));
    for (int it = 0; it < iters; ++it) {
      const uint32_t acc = it == 0 ? 0u : 1u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(id), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&mbar)));
  }
  uint32_t done = 0;
  for (uint32_t k = 0; k < kTcWait && !done; ++k)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(su32(&mbar)), "r"(0u));
  if (!done && tid == 0) atomicCAS(status, 0, (int)QRKIT_ETIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}

}  // namespace
}  // namespace qrkit

extern "C" qrkit_status qrkit_peak_probe(int device, int kind, double* tflops) {
  using namespace qrkit;
  if (!tflops || kind < 0 || kind > 2) return QRKIT_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return QRKIT_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return QRKIT_ECUDA;
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  void* buf = nullptr;
  qrkit_status rc = QRKIT_OK;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaMalloc(&buf, 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 64, st);
  double flops = 0.0;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
    if ((e = cudaEventRecord(a, st)) != cudaSuccess) break;
    if (kind == 0 || kind == 1) {
      const int blocks = sms * 8, iters = kind == 0 ? 8192 : 1024;
      if (kind == 0)
        fma_probe_kernel<float><<<blocks, kFmaThreads, 0, st>>>(1.0f, iters, (float*)buf);
      else
        fma_probe_kernel<double><<<blocks, kFmaThreads, 0, st>>>(1.0, iters, (double*)buf);
      flops = 2.0 * kChains * (double)iters * kFmaThreads * blocks;
    } else {
      const int iters = 4096;
      const size_t smem = kTcSmem;
      e = cudaFuncSetAttribute(tf32_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) break;
      tf32_probe_kernel<<<sms, kTcThreads, smem, st>>>(iters, (int*)buf);
      flops = 2.0 * 128.0 * kTcN * 8.0 * iters * sms;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    e = cudaEventRecord(b, st);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&status, buf, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = QRKIT_ECUDA;
  else if (kind == 2 && status != 0) rc = (qrkit_status)status;
  else *tflops = flops / (ms * 1e-3) / 1e12;
  if (buf) cudaFree(buf);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  cudaSetDevice(prev);
  return rc;
}

namespace qrkit {
namespace {

// Streams `n16` 16-byte words from src (pinned host memory, read by the GPU over the host link)
// into dst (device memory): the rate a kernel that reads its inputs straight from the host gets.
__global__ void __launch_bounds__(256) host_read_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                        int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
}

}  // namespace
}  // namespace qrkit

extern "C" qrkit_status qrkit_host_link_probe(int device, int64_t bytes, double* copy_gbs, double* kernel_gbs) {
  using namespace qrkit;
  if (!copy_gbs || !kernel_gbs || bytes < (1 << 20) || (bytes & 15)) return QRKIT_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return QRKIT_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return QRKIT_ECUDA;
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  void *h = nullptr, *d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaHostAlloc(&h, (size_t)bytes, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e == cudaSuccess) e = cudaMalloc(&d, (size_t)bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) memset(h, 1, (size_t)bytes);
  void* hd = nullptr;
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&hd, h, 0);
  float ms_copy = 0.f, ms_kernel = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first of each runs warms up
    if ((e = cudaEventRecord(a, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d, h, (size_t)bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaEventRecord(b, st)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    e = cudaEventElapsedTime(&ms_copy, a, b);
  }
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    if ((e = cudaEventRecord(a, st)) != cudaSuccess) break;
    host_read_kernel<<<sms * 8, 256, 0, st>>>((const uint4*)hd, (uint4*)d, bytes / 16);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaEventRecord(b, st)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    e = cudaEventElapsedTime(&ms_kernel, a, b);
  }
  if (e == cudaSuccess) {
    *copy_gbs = (double)bytes / (ms_copy * 1e-3) / 1e9;
    *kernel_gbs = (double)bytes / (ms_kernel * 1e-3) / 1e9;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  if (d) cudaFree(d);
  if (h) cudaFreeHost(h);
  cudaSetDevice(prev);
  return e == cudaSuccess ? QRKIT_OK : QRKIT_ECUDA;
}
