// Batched requests: the users x ads inner products on the tensor cores
// (tcgen05.mma fed by tensor TMA, accumulators in TMEM), plus the tensor-map
// plumbing they need.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ebr_internal.cuh"
#include "ebr_umma.cuh"

namespace ebr {

// --------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static int get_encoder() {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (g_encode) return EBR_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    set_error("cuTensorMapEncodeTiled unavailable: %s", cudaGetErrorString(e));
    return EBR_ECUDA;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return EBR_OK;
}

// Row-major [rows][cols] BF16 matrix viewed as a 2-D tensor, boxes of
// 64 columns x box_rows rows, 128-byte swizzle (the UMMA K-major layout).
int make_tmap_bf16(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                   uint32_t box_rows) {
  EBR_TRY(get_encoder());
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for %llu x %llu, box %u", (int)r,
              (unsigned long long)rows, (unsigned long long)cols, box_rows);
    return EBR_ECUDA;
  }
  return EBR_OK;
}

// ------------------------------------------------------------ GEMM check
// out[i][b] = sum_t A[i][t] * U[b][t] for one 128-row tile per CTA: the
// tensor-core building block of the batched scan, exposed for testing.
__global__ void __launch_bounds__(128) k_gemm_bf16(const __grid_constant__ CUtensorMap ma,
                                                   const __grid_constant__ CUtensorMap mu,
                                                   uint32_t n, uint32_t B, uint32_t d,
                                                   float *__restrict__ out,
                                                   uint32_t *__restrict__ flags) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base, ok;
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t kb_n = d / 64;
  uint8_t *sa = smem;                        // kb_n x [128 rows x 128 B]
  uint8_t *su = smem + (size_t)kb_n * 16384;  // kb_n x [B rows x 128 B]
  const int warp = threadIdx.x >> 5;
  uint32_t ncols = 32;
  while (ncols < B) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_base, ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    fence_mbar_init();
    ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t row0 = blockIdx.x * 128;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar_tma, kb_n * (16384u + B * 128u));
    for (uint32_t kb = 0; kb < kb_n; kb++) {
      tma_load_2d(sa + kb * 16384, &ma, (int)(kb * 64), (int)row0, &bar_tma);
      tma_load_2d(su + (size_t)kb * B * 128, &mu, (int)(kb * 64), 0, &bar_tma);
    }
    if (!mbar_wait_bounded(&bar_tma, 0, kWaitTimeoutNs)) {
      ok = 0;
      atomicOr(flags, DEVERR_TIMEOUT);
    } else {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16_f32(128, B);
      for (uint32_t k = 0; k < d / 16; k++) {
        const uint32_t kb = k / 4, kk = k % 4;
        const uint64_t ad = sdesc_k_sw128(smem_u32(sa + kb * 16384 + kk * 32));
        const uint64_t bd = sdesc_k_sw128(smem_u32(su + (size_t)kb * B * 128 + kk * 32));
        umma_bf16(tmem_base, ad, bd, idesc, k > 0 ? 1u : 0u);
      }
      umma_commit(&bar_mma);
      if (!mbar_wait_bounded(&bar_mma, 0, kWaitTimeoutNs)) {
        ok = 0;
        atomicOr(flags, DEVERR_TIMEOUT);
      }
    }
  }
  __syncthreads();
  tc_fence_after();
  if (ok) {
    mbar_try_wait(&bar_mma, 0);
    const uint32_t row = row0 + warp * 32 + (threadIdx.x & 31);
    for (uint32_t c = 0; c < B / 32; c++) {
      uint32_t r[32];
      tmem_ld32(tmem_base + ((uint32_t)(warp * 32) << 16) + c * 32, r);
      tmem_ld_wait();
      if (row < n)
        for (int j = 0; j < 32; j++) out[(uint64_t)row * B + c * 32 + j] = __uint_as_float(r[j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_base, ncols);
}

}  // namespace ebr

using namespace ebr;

extern "C" int ebr_debug_gemm_bf16(const uint16_t *A, uint32_t n, const uint16_t *U, uint32_t B,
                                   uint32_t d, float *out, void *stream) {
  clear_error();
  if (!A || !U || !out || n == 0 || (d != 64 && d != 128) || B < 32 || B > 256 || B % 32) {
    set_error("ebr_debug_gemm_bf16: need d in {64, 128}, B a multiple of 32 in 32..256");
    return EBR_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  CUtensorMap ma, mu;
  EBR_TRY(make_tmap_bf16(&ma, A, n, d, 128));
  EBR_TRY(make_tmap_bf16(&mu, U, B, d, B));
  uint32_t *flags = nullptr;
  EBR_CUDA_TRY(cudaMallocAsync((void **)&flags, 4, st));
  EBR_CUDA_TRY(cudaMemsetAsync(flags, 0, 4, st));
  const size_t smem = 1024 + (size_t)(d / 64) * (16384 + B * 128);
  EBR_CUDA_TRY(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  k_gemm_bf16<<<(n + 127) / 128, 128, smem, st>>>(ma, mu, n, B, d, out, flags);
  EBR_CUDA_TRY(cudaGetLastError());
  uint32_t hf = 0;
  EBR_CUDA_TRY(cudaMemcpyAsync(&hf, flags, 4, cudaMemcpyDeviceToHost, st));
  EBR_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(flags, st);
  return check_device_flags(hf, "ebr_debug_gemm_bf16");
}
