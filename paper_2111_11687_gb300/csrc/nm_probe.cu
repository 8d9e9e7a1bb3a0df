// Ceilings of this GPU that the transport's roofline is quoted against: the
// L2 read bandwidth for a working set that stays in the L2, and the rate of
// scattered 64-bit atomic adds whose results are unused (the reduction form
// the tally deposits compile to).  Neither figure is published for the
// GB300, so both are measured here with CUDA events.
#include <cstdarg>
#include <cstdio>

#include "nm_internal.cuh"

using namespace nm;

namespace {

nm_status fail(nm_status st, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error_message(buf);
  return st;
}

// Every thread streams 16-byte words of the buffer `reps` times with L2-only
// loads (no L1 allocation), four independent loads in flight per iteration.
// The XOR of what it read goes to `sink` only on an impossible value, which
// keeps the loads without a store per thread.
__global__ void l2_read_kernel(const uint4* __restrict__ buf, int64_t n16, int reps, uint32_t* sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int r = 0; r < reps; ++r) {
    int64_t i = t;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                  d = __ldcg(buf + i + 3 * stride);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    for (; i < n16; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
    acc += (uint32_t)r;
  }
  if (acc == 0x9E3779B9u) sink[t & 1023] = acc;
}

// Scattered atomic adds: every thread adds 1 to `per_thread` slots chosen by
// a 32-bit xorshift generator, masked to the buffer's power-of-two size.
__global__ void atomic_add_kernel(ull* buf, uint32_t mask, int per_thread) {
  uint32_t x = ((uint32_t)(blockIdx.x * blockDim.x + threadIdx.x) + 1u) * 0x9E3779B9u;
  for (int k = 0; k < per_thread; ++k) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    atomicAdd(buf + (x & mask), 1ull);
  }
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

int sms_of_current_device() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

}  // namespace

extern "C" nm_status nm_probe_l2_read(int64_t bytes, int32_t reps, double* gb_per_s) {
  if (!gb_per_s || bytes < (1 << 20) || bytes > ((int64_t)1 << 31) || (bytes & 15) || reps < 1 || reps > 1000)
    return fail(NM_ERR_ARG, "nm_probe_l2_read: 1 MiB <= bytes <= 2 GiB (multiple of 16), 1 <= reps <= 1000");
  const int sms = sms_of_current_device();
  if (sms <= 0) return fail(NM_ERR_CUDA, "nm_probe_l2_read: no device");
  uint4* buf = nullptr;
  uint32_t* sink = nullptr;
  cudaStream_t s = nullptr;
  Timer tm;
  float ms = 0.0f;
  cudaError_t e = cudaMalloc(&buf, bytes);
  if (!e) e = cudaMalloc(&sink, 1024 * sizeof(uint32_t));
  if (!e) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (!e) e = cudaMemsetAsync(buf, 0x5a, bytes, s);
  if (!e) e = cudaEventCreate(&tm.a);
  if (!e) e = cudaEventCreate(&tm.b);
  const int64_t n16 = bytes / 16;
  const int grid = sms * 8, block = 256;
  if (!e) {
    l2_read_kernel<<<grid, block, 0, s>>>(buf, n16, 2, sink);   // brings the buffer into the L2
    e = cudaGetLastError();
  }
  if (!e) e = cudaEventRecord(tm.a, s);
  if (!e) {
    l2_read_kernel<<<grid, block, 0, s>>>(buf, n16, reps, sink);
    e = cudaGetLastError();
  }
  if (!e) e = cudaEventRecord(tm.b, s);
  if (!e) e = cudaEventSynchronize(tm.b);
  if (!e) e = cudaEventElapsedTime(&ms, tm.a, tm.b);
  if (s) cudaStreamDestroy(s);
  cudaFree(buf);
  cudaFree(sink);
  if (e) return fail(NM_ERR_CUDA, "nm_probe_l2_read: %s", cudaGetErrorString(e));
  *gb_per_s = (double)bytes * reps / (ms * 1e-3) / 1e9;
  return NM_OK;
}

extern "C" nm_status nm_probe_atomic_add_u64(int64_t slots, int64_t ops, double* ops_per_s) {
  if (!ops_per_s || slots < 1024 || slots > ((int64_t)1 << 28) || (slots & (slots - 1)) || ops < (1 << 20) ||
      ops > ((int64_t)1 << 34))
    return fail(NM_ERR_ARG, "nm_probe_atomic_add_u64: slots a power of two in [2^10, 2^28], 2^20 <= ops <= 2^34");
  const int sms = sms_of_current_device();
  if (sms <= 0) return fail(NM_ERR_CUDA, "nm_probe_atomic_add_u64: no device");
  const int grid = sms * 8, block = 256;
  const int64_t threads = (int64_t)grid * block;
  const int per_thread = (int)((ops + threads - 1) / threads);
  ull* buf = nullptr;
  cudaStream_t s = nullptr;
  Timer tm;
  float ms = 0.0f;
  cudaError_t e = cudaMalloc(&buf, slots * sizeof(ull));
  if (!e) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (!e) e = cudaMemsetAsync(buf, 0, slots * sizeof(ull), s);
  if (!e) e = cudaEventCreate(&tm.a);
  if (!e) e = cudaEventCreate(&tm.b);
  if (!e) {
    atomic_add_kernel<<<grid, block, 0, s>>>(buf, (uint32_t)(slots - 1), per_thread > 8 ? 8 : per_thread);
    e = cudaGetLastError();
  }
  if (!e) e = cudaEventRecord(tm.a, s);
  if (!e) {
    atomic_add_kernel<<<grid, block, 0, s>>>(buf, (uint32_t)(slots - 1), per_thread);
    e = cudaGetLastError();
  }
  if (!e) e = cudaEventRecord(tm.b, s);
  if (!e) e = cudaEventSynchronize(tm.b);
  if (!e) e = cudaEventElapsedTime(&ms, tm.a, tm.b);
  if (s) cudaStreamDestroy(s);
  cudaFree(buf);
  if (e) return fail(NM_ERR_CUDA, "nm_probe_atomic_add_u64: %s", cudaGetErrorString(e));
  *ops_per_s = (double)threads * per_thread / (ms * 1e-3);
  return NM_OK;
}
