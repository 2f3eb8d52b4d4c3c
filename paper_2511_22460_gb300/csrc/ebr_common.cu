// Error state, device buffers and the BF16 / FP8-e4m3 converters.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstring>
#include <mutex>

#include "ebr_internal.cuh"

namespace ebr {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

void clear_error() { g_err.clear(); }

int check_device_flags(uint32_t flags, const char *where) {
  if (!flags) return EBR_OK;
  if (flags & DEVERR_TIMEOUT) {
    set_error("%s: a bounded device wait timed out (flags 0x%x)", where, flags);
    return EBR_ETIMEDOUT;
  }
  set_error("%s: device-side input check failed (flags 0x%x: %s%s%s%s%s%s)", where, flags,
            (flags & DEVERR_BAD_KEY) ? "query key >= n_keys " : "",
            (flags & DEVERR_BAD_AD) ? "ad id >= n_ads " : "",
            (flags & DEVERR_BAD_USER) ? "user value >= vocabulary " : "",
            (flags & DEVERR_OVERFLOW) ? "capacity overflow " : "",
            (flags & DEVERR_BAD_BUILD_KEY) ? "key >= n_keys " : "",
            (flags & DEVERR_RANGE) ? "a non-finite query weight " : "");
  return EBR_EDATA;
}

int dev_alloc(DevBuf &b, size_t bytes) {
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return EBR_ENOMEM;
  }
  b.bytes = bytes;
  return EBR_OK;
}

void dev_free(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

int dev_reserve(DevBuf &b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return EBR_OK;
  dev_free(b);
  return dev_alloc(b, bytes);
}

// ----------------------------------------------------------- converters
__global__ void k_to_bf16(const float *__restrict__ x, uint64_t n, uint16_t *__restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 h = __float2bfloat16_rn(x[i]);
    out[i] = *reinterpret_cast<uint16_t *>(&h);
  }
}

__global__ void k_to_e4m3(const float *__restrict__ x, uint64_t n, uint8_t *__restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint8_t)__nv_cvt_float_to_fp8(x[i], __NV_SATFINITE, __NV_E4M3);
}

// Per-row FP8 quantisation: scale = max|x| / 448 (1 for an all-zero row),
// code = E4M3(x / scale), saturating.  One warp per row.
__global__ void k_rows_to_e4m3(const float *__restrict__ x, uint64_t n, uint32_t d,
                               uint8_t *__restrict__ q, float *__restrict__ scale) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < n; r += nwarps) {
    const float *row = x + r * d;
    float mx = 0.f;
    for (uint32_t t = lane; t < d; t += 32) mx = fmaxf(mx, fabsf(row[t]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float sc = mx > 0.f ? __fdiv_rn(mx, 448.0f) : 1.0f;
    if (lane == 0) scale[r] = sc;
    for (uint32_t t = lane; t < d; t += 32)
      q[r * d + t] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(row[t], sc), __NV_SATFINITE,
                                                    __NV_E4M3);
  }
}

int launch_quantize(const float *x, uint64_t n, ebr_dtype dt, void *out, cudaStream_t st) {
  if (n == 0) return EBR_OK;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  if (dt == EBR_BF16)
    k_to_bf16<<<blocks, 256, 0, st>>>(x, n, (uint16_t *)out);
  else if (dt == EBR_FP8E4M3)
    k_to_e4m3<<<blocks, 256, 0, st>>>(x, n, (uint8_t *)out);
  else {
    set_error("quantize: dtype must be BF16 or FP8E4M3");
    return EBR_EINVAL;
  }
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

int launch_quantize_rows_fp8(const float *x, uint64_t n, uint32_t d, uint8_t *q, float *scale,
                             cudaStream_t st) {
  if (n == 0) return EBR_OK;
  uint64_t warps = n;
  int blocks = (int)((warps * 32 + 255) / 256);
  if (blocks > 16384) blocks = 16384;
  k_rows_to_e4m3<<<blocks, 256, 0, st>>>(x, n, d, q, scale);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

}  // namespace ebr

extern "C" const char *ebr_last_error(void) { return ebr::g_err.c_str(); }

extern "C" int ebr_version(void) { return 0x000100; }

extern "C" int ebr_quantize(const float *x, uint64_t n, ebr_dtype dtype, void *out,
                            void *stream) {
  ebr::clear_error();
  if ((!x || !out) && n) {
    ebr::set_error("ebr_quantize: null pointer");
    return EBR_EINVAL;
  }
  return ebr::launch_quantize(x, n, dtype, out, (cudaStream_t)stream);
}
