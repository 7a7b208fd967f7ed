// Memory-bound helpers of the learned network and of whole-volume inference:
//   leaky ReLU on SH activations (between LSC layers) and its adjoint,
//   brain-mask compaction (voxel index list, ascending, deterministic),
//   gather / scatter of voxel columns between a volume and its masked list.
#include <cuda_runtime.h>

#include "../../include/delimit.h"
#include "kernels.h"

namespace delimit {

__device__ __forceinline__ float ld1(const float* p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st1(float* p, float v) { *p = v; }
__device__ __forceinline__ void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <typename T>
__global__ void leaky_kernel(const T* x, T* y, int64_t rows, int64_t n, int64_t ldx,
                             int64_t ldy, float slope) {
  const int64_t r = blockIdx.y;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float a = ld1(x + r * ldx + v);
    st1(y + r * ldy + v, a > 0.f ? a : slope * a);
  }
}

// 16-byte vectors of BF16 (rows 16-byte aligned); one grid row per feature row
__global__ void leaky_bf16x8_kernel(const __nv_bfloat16* x, __nv_bfloat16* y, int64_t n, int64_t ldx, int64_t ldy,
                                    float slope) {
  const int64_t r = blockIdx.y;
  const int64_t n8 = n / 8;
  const uint4* xr = reinterpret_cast<const uint4*>(x + r * ldx);
  uint4* yr = reinterpret_cast<uint4*>(y + r * ldy);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n8; v += (int64_t)gridDim.x * blockDim.x) {
    uint4 u = xr[v];
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(h[i]);
      f.x = f.x > 0.f ? f.x : slope * f.x;
      f.y = f.y > 0.f ? f.y : slope * f.y;
      h[i] = __float22bfloat162_rn(f);
    }
    yr[v] = u;
  }
  for (int64_t v = n8 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float a = __bfloat162float(x[r * ldx + v]);
    y[r * ldy + v] = __float2bfloat16_rn(a > 0.f ? a : slope * a);
  }
}

__global__ void leaky_bwd_bf16x8_kernel(const __nv_bfloat16* __restrict__ y, const __nv_bfloat16* __restrict__ dy,
                                        __nv_bfloat16* __restrict__ dx, int64_t n, int64_t ldy, int64_t lddy,
                                        int64_t lddx, float slope) {
  const int64_t r = blockIdx.y;
  const int64_t n8 = n / 8;
  const uint4* yr = reinterpret_cast<const uint4*>(y + r * ldy);
  const uint4* gr = reinterpret_cast<const uint4*>(dy + r * lddy);
  uint4* dr = reinterpret_cast<uint4*>(dx + r * lddx);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n8; v += (int64_t)gridDim.x * blockDim.x) {
    const uint4 uy = yr[v];
    uint4 ug = gr[v];
    const __nv_bfloat162* hy = reinterpret_cast<const __nv_bfloat162*>(&uy);
    __nv_bfloat162* hg = reinterpret_cast<__nv_bfloat162*>(&ug);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 a = __bfloat1622float2(hy[i]);
      float2 g = __bfloat1622float2(hg[i]);
      g.x = a.x > 0.f ? g.x : slope * g.x;
      g.y = a.y > 0.f ? g.y : slope * g.y;
      hg[i] = __float22bfloat162_rn(g);
    }
    dr[v] = ug;
  }
  for (int64_t v = n8 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float a = __bfloat162float(y[r * ldy + v]), g = __bfloat162float(dy[r * lddy + v]);
    dx[r * lddx + v] = __float2bfloat16_rn(a > 0.f ? g : slope * g);
  }
}

static bool al16(const void* p, int64_t ld) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (ld * 2) % 16 == 0;
}

// dx = dy * (y > 0 ? 1 : slope): the forward output y carries the sign of its input
template <typename T>
__global__ void leaky_bwd_kernel(const T* __restrict__ y, const T* __restrict__ dy, T* __restrict__ dx, int64_t rows,
                                 int64_t n, int64_t ldy, int64_t lddy, int64_t lddx, float slope) {
  const int64_t r = blockIdx.y;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float a = ld1(y + r * ldy + v), g = ld1(dy + r * lddy + v);
    st1(dx + r * lddx + v, a > 0.f ? g : slope * g);
  }
}

// ---- mask compaction: per-block counts, one-block scan, ordered writes ----
constexpr int kCompactBlock = 256, kCompactPer = 16;  // elements per block = 4096

__global__ void compact_count_kernel(const uint8_t* __restrict__ mask, int64_t n, int64_t* __restrict__ counts) {
  __shared__ int64_t part[kCompactBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kCompactBlock * kCompactPer;
  int c = 0;
  for (int i = 0; i < kCompactPer; ++i) {
    const int64_t idx = base + (int64_t)i * kCompactBlock + threadIdx.x;
    c += (idx < n && mask[idx]) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (threadIdx.x % 32 == 0) part[threadIdx.x / 32] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kCompactBlock / 32; ++w) t += part[w];
    counts[blockIdx.x] = t;
  }
}

// exclusive scan of counts[nb] in place, total to *total (one block, sequential chunks)
__global__ void compact_scan_kernel(int64_t* __restrict__ counts, int64_t nb, int64_t* __restrict__ total) {
  __shared__ int64_t buf[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
    const int64_t i = c0 + threadIdx.x;
    const int64_t v = i < nb ? counts[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan
      const int64_t t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) counts[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void compact_write_kernel(const uint8_t* __restrict__ mask, int64_t n, const int64_t* __restrict__ offs,
                                     int64_t* __restrict__ out) {
  __shared__ int wsum[kCompactBlock / 32];
  __shared__ int64_t run;
  const int64_t base = (int64_t)blockIdx.x * kCompactBlock * kCompactPer;
  if (threadIdx.x == 0) run = offs[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int i = 0; i < kCompactPer; ++i) {
    const int64_t idx = base + (int64_t)i * kCompactBlock + threadIdx.x;
    const bool on = idx < n && mask[idx];
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int64_t wbase = run;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    if (on) out[wbase + before] = idx;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t t = 0;
      for (int w = 0; w < kCompactBlock / 32; ++w) t += wsum[w];
      run += t;
    }
    __syncthreads();
  }
}

// out-of-range indices are skipped (gather writes 0), never dereferenced
template <typename T>
__global__ void gather_kernel(const T* __restrict__ src, int64_t ld_src, int64_t n_src, const int64_t* __restrict__ idx,
                              int64_t n, T* __restrict__ dst, int64_t ld_dst) {
  const int64_t r = blockIdx.y;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx[j];
    dst[r * ld_dst + j] = (k >= 0 && k < n_src) ? src[r * ld_src + k] : T(0.f);
  }
}

template <typename T>
__global__ void scatter_kernel(const T* __restrict__ src, int64_t ld_src, const int64_t* __restrict__ idx, int64_t n,
                               T* __restrict__ dst, int64_t ld_dst, int64_t n_dst) {
  const int64_t r = blockIdx.y;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx[j];
    if (k >= 0 && k < n_dst) dst[r * ld_dst + k] = src[r * ld_src + j];
  }
}

static unsigned grid_x(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 1024) g = 1024;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace delimit

using namespace delimit;

static bool ok_rows(int64_t rows) { return rows >= 1 && rows <= 65535; }

// argument refusal with its reason for delimit_last_error()
static delimit_status bad_arg(const char* fn, const char* what) {
  set_last_error(std::string(fn) + ": " + what);
  return DELIMIT_ERR_INVALID_ARG;
}

// status of the launches just made, with the CUDA error text on failure
static delimit_status launch_status(const char* fn) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return DELIMIT_OK;
  set_last_error(std::string(fn) + ": " + cudaGetErrorString(e));
  return DELIMIT_ERR_CUDA;
}

static const char* kActArgs = "need non-NULL pointers, 1 <= rows <= 65535, ld >= n_vox and dtype F32 or BF16";

extern "C" {

delimit_status delimit_leaky_relu(const void* x, void* y, int64_t rows, int64_t n_vox, int64_t ld_x, int64_t ld_y,
                                  float slope, delimit_dtype t, void* stream) {
  if (n_vox == 0) return DELIMIT_OK;
  if (!x || !y || n_vox < 0 || !ok_rows(rows) || ld_x < n_vox || ld_y < n_vox || (t != DELIMIT_F32 && t != DELIMIT_BF16))
    return bad_arg("delimit_leaky_relu", kActArgs);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid(grid_x(n_vox), (unsigned)rows);
  if (t == DELIMIT_F32) {
    leaky_kernel<float><<<grid, 256, 0, st>>>((const float*)x, (float*)y, rows, n_vox, ld_x, ld_y, slope);
  } else if (al16(x, ld_x) && al16(y, ld_y)) {
    dim3 g8(grid_x((n_vox + 7) / 8), (unsigned)rows);
    leaky_bf16x8_kernel<<<g8, 256, 0, st>>>((const __nv_bfloat16*)x, (__nv_bfloat16*)y, n_vox, ld_x, ld_y, slope);
  } else {
    leaky_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)x, (__nv_bfloat16*)y, rows, n_vox, ld_x,
                                                      ld_y, slope);
  }
  count_launch();
  return launch_status("delimit_leaky_relu");
}

delimit_status delimit_leaky_relu_backward(const void* y, const void* dy, void* dx, int64_t rows, int64_t n_vox,
                                           int64_t ld_y, int64_t ld_dy, int64_t ld_dx, float slope, delimit_dtype t,
                                           void* stream) {
  if (n_vox == 0) return DELIMIT_OK;
  if (!y || !dy || !dx || n_vox < 0 || !ok_rows(rows) || ld_y < n_vox || ld_dy < n_vox || ld_dx < n_vox ||
      (t != DELIMIT_F32 && t != DELIMIT_BF16))
    return bad_arg("delimit_leaky_relu_backward", kActArgs);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid(grid_x(n_vox), (unsigned)rows);
  if (t == DELIMIT_F32) {
    leaky_bwd_kernel<float><<<grid, 256, 0, st>>>((const float*)y, (const float*)dy, (float*)dx, rows, n_vox, ld_y,
                                                  ld_dy, ld_dx, slope);
  } else if (al16(y, ld_y) && al16(dy, ld_dy) && al16(dx, ld_dx)) {
    dim3 g8(grid_x((n_vox + 7) / 8), (unsigned)rows);
    leaky_bwd_bf16x8_kernel<<<g8, 256, 0, st>>>((const __nv_bfloat16*)y, (const __nv_bfloat16*)dy, (__nv_bfloat16*)dx,
                                                n_vox, ld_y, ld_dy, ld_dx, slope);
  } else {
    leaky_bwd_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)y, (const __nv_bfloat16*)dy,
                                                          (__nv_bfloat16*)dx, rows, n_vox, ld_y, ld_dy, ld_dx, slope);
  }
  count_launch();
  return launch_status("delimit_leaky_relu_backward");
}

size_t delimit_mask_compact_workspace_size(int64_t n) {
  if (n < 0) return 0;
  const int64_t nb = (n + kCompactBlock * kCompactPer - 1) / (kCompactBlock * kCompactPer);
  return (size_t)(nb + 1) * sizeof(int64_t) + 256;
}

delimit_status delimit_mask_compact(const uint8_t* mask, int64_t n, int64_t* index, int64_t* count, void* workspace,
                                    size_t ws_bytes, void* stream) {
  if (n < 0 || !count || (n > 0 && (!mask || !index)))
    return bad_arg("delimit_mask_compact", "need n >= 0, count non-NULL, and mask and index non-NULL when n > 0");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) return DELIMIT_OK;
    set_last_error(std::string("delimit_mask_compact: ") + cudaGetErrorString(e));
    return DELIMIT_ERR_CUDA;
  }
  if (ws_bytes < delimit_mask_compact_workspace_size(n) || !workspace) {
    set_last_error("delimit_mask_compact: workspace NULL or smaller than delimit_mask_compact_workspace_size(n)");
    return DELIMIT_ERR_WORKSPACE;
  }
  const int64_t nb = (n + kCompactBlock * kCompactPer - 1) / (kCompactBlock * kCompactPer);
  int64_t* counts = static_cast<int64_t*>(workspace);
  compact_count_kernel<<<(unsigned)nb, kCompactBlock, 0, st>>>(mask, n, counts);
  count_launch();
  compact_scan_kernel<<<1, 1024, 0, st>>>(counts, nb, count);
  count_launch();
  compact_write_kernel<<<(unsigned)nb, kCompactBlock, 0, st>>>(mask, n, counts, index);
  count_launch();
  return launch_status("delimit_mask_compact");
}

delimit_status delimit_gather_voxels(const void* src, int64_t ld_src, int64_t n_src, int64_t rows, const int64_t* index,
                                     int64_t n, void* dst, int64_t ld_dst, delimit_dtype t, void* stream) {
  if (n == 0) return DELIMIT_OK;
  if (!src || !dst || !index || n < 0 || n_src < 0 || ld_src < n_src || !ok_rows(rows) || ld_dst < n ||
      (t != DELIMIT_F32 && t != DELIMIT_BF16))
    return bad_arg("delimit_gather_voxels",
                   "need non-NULL pointers, n >= 0, 0 <= n_src <= ld_src, n <= ld_dst, 1 <= rows <= 65535, F32 or BF16");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid(grid_x(n), (unsigned)rows);
  if (t == DELIMIT_F32)
    gather_kernel<float><<<grid, 256, 0, st>>>((const float*)src, ld_src, n_src, index, n, (float*)dst, ld_dst);
  else
    gather_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)src, ld_src, n_src, index, n,
                                                       (__nv_bfloat16*)dst, ld_dst);
  count_launch();
  return launch_status("delimit_gather_voxels");
}

delimit_status delimit_scatter_voxels(const void* src, int64_t ld_src, int64_t rows, const int64_t* index, int64_t n,
                                      void* dst, int64_t ld_dst, int64_t n_dst, delimit_dtype t, void* stream) {
  if (n == 0) return DELIMIT_OK;
  if (!src || !dst || !index || n < 0 || n_dst < 0 || ld_dst < n_dst || !ok_rows(rows) || ld_src < n ||
      (t != DELIMIT_F32 && t != DELIMIT_BF16))
    return bad_arg("delimit_scatter_voxels",
                   "need non-NULL pointers, n >= 0, 0 <= n_dst <= ld_dst, n <= ld_src, 1 <= rows <= 65535, F32 or BF16");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid(grid_x(n), (unsigned)rows);
  if (t == DELIMIT_F32)
    scatter_kernel<float><<<grid, 256, 0, st>>>((const float*)src, ld_src, index, n, (float*)dst, ld_dst, n_dst);
  else
    scatter_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)src, ld_src, index, n,
                                                        (__nv_bfloat16*)dst, ld_dst, n_dst);
  count_launch();
  return launch_status("delimit_scatter_voxels");
}

}  // extern "C"
