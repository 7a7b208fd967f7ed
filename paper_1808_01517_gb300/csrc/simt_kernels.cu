// CUDA-core kernels of the spherical layers: the FP32 accurate path of every
// step, and the small weight-side steps of the BF16 path.
//
//   transform_simt   grouped Signal2SH / SH2Signal and their adjoints (Sec. 2.2)
//   build_w          collapsed LSC operator W = sum_k w_k M_{s,k} per shell pair (Sec. 2.3)
//   row_gemm_simt    LSC forward / input-gradient GEMM over voxels
//   wgrad_simt       LSC weight-gradient GEMM (reduction over voxels, split, deterministic)
//   reduce_dw        dW -> kernel-point weights dw and bias gradient db
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "kernels.h"

namespace delimit {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

__device__ __forceinline__ float ldf(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------
// Grouped transform: one thread owns VPT voxels and OPT output rows.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, int OPT, int VPT>
__global__ void __launch_bounds__(128) transform_simt_kernel(const __grid_constant__ TransformArgs a, int ochunks) {
  constexpr int KC = 32;
  __shared__ __align__(16) float Ts[KC][OPT];
  const TransformGroup& gd = a.g[blockIdx.z];
  const int c = blockIdx.y / ochunks, oc = blockIdx.y % ochunks;
  const int o0 = oc * OPT;
  if (o0 >= gd.n_out) return;
  const int no = min(OPT, gd.n_out - o0);
  int64_t v[VPT];
  bool ok[VPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    v[k] = (int64_t)blockIdx.x * (128 * VPT) + threadIdx.x + k * 128;
    ok[k] = v[k] < a.n_vox;
  }
  float acc[OPT][VPT];
#pragma unroll
  for (int o = 0; o < OPT; ++o)
#pragma unroll
    for (int k = 0; k < VPT; ++k) acc[o][k] = 0.f;
  const Tin* X = reinterpret_cast<const Tin*>(a.X) + (gd.x_row0 + (int64_t)c * gd.x_cstride) * a.ldx;
  for (int j0 = 0; j0 < gd.n_in; j0 += KC) {
    const int nj = min(KC, gd.n_in - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * OPT; idx += 128) {
      const int jj = idx / OPT, oo = idx % OPT;
      Ts[jj][oo] = (jj < nj && oo < no) ? gd.T[(int64_t)(o0 + oo) * gd.n_in + j0 + jj] : 0.f;
    }
    __syncthreads();
    for (int jj = 0; jj < nj; ++jj) {
      const Tin* xr = X + (int64_t)(j0 + jj) * a.ldx;
      float x[VPT];
#pragma unroll
      for (int k = 0; k < VPT; ++k) x[k] = ok[k] ? ldf(xr + v[k]) : 0.f;
#pragma unroll
      for (int o = 0; o < OPT; o += 4) {
        const float4 t = *reinterpret_cast<const float4*>(&Ts[jj][o]);
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          acc[o][k] = fmaf(t.x, x[k], acc[o][k]);
          acc[o + 1][k] = fmaf(t.y, x[k], acc[o + 1][k]);
          acc[o + 2][k] = fmaf(t.z, x[k], acc[o + 2][k]);
          acc[o + 3][k] = fmaf(t.w, x[k], acc[o + 3][k]);
        }
      }
    }
  }
  Tout* Y = reinterpret_cast<Tout*>(a.Y) + (gd.y_row0 + (int64_t)c * gd.y_cstride + o0) * a.ldy;
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    if (o < no) {
#pragma unroll
      for (int k = 0; k < VPT; ++k)
        if (ok[k]) stf(Y + (int64_t)o * a.ldy + v[k], acc[o][k]);
    }
  }
}

// ---------------------------------------------------------------------------
// Grouped transform with staged tiles (n_in, n_out <= 120).  A persistent block
// walks tiles (group, channel, 128 voxels); the group's operator T^T
// [n_in][12 x OG] stays in shared memory while the group lasts, each tile's
// input rows [n_in][128 voxels] arrive by cp.async (all rows in flight at once).
// Thread (q, og) computes 4 voxels (4q..4q+3) x 12 outputs: per input row one
// vector load of x, three of T^T, 48 FMAs.  A warp holds 32 consecutive voxel
// quads of one output group, so every output row is one 512-byte (FP32) run.
// ---------------------------------------------------------------------------
constexpr int kTfVox = 128, kTfOpt = 12, kTfMaxOut = 120;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ float4 ld_x4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld_x4(const __nv_bfloat16* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                     __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ void st_y4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st_y4(__nv_bfloat16* p, float a, float b, float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&lo);
  u.y = *reinterpret_cast<uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(p) = u;
}

// GATHER: output voxel v reads input column a.index[v] scaled by 1 / a.b0[index[v]]
// (plain loads into an FP32 tile: columns are not contiguous).
template <typename Tin, typename Tout, bool GATHER>
__global__ void __launch_bounds__(32 * (kTfMaxOut / kTfOpt)) transform_staged_kernel(const __grid_constant__ TransformArgs a,
                                                                                     int n_groups, int og_count,
                                                                                     int max_in) {
  using Ts = typename std::conditional<GATHER, float, Tin>::type;  // type of the staged input tile
  extern __shared__ float4 tf_smem4[];
  float* Tt = reinterpret_cast<float*>(tf_smem4);                 // [max_in][12 * og_count]
  Ts* Xs = reinterpret_cast<Ts*>(Tt + max_in * kTfOpt * og_count);  // [max_in][128]
  int64_t* sidx = reinterpret_cast<int64_t*>(Xs + max_in * kTfVox);  // GATHER: source column per voxel
  float* sinv = reinterpret_cast<float*>(sidx + kTfVox);            // GATHER: 1 / b0 per voxel
  const int ldt = kTfOpt * og_count;
  const int tid = threadIdx.x, q = tid % 32, og = tid / 32;
  const int64_t vt_count = (a.n_vox + kTfVox - 1) / kTfVox;
  const int64_t per_group = vt_count * a.channels;
  const int64_t total = per_group * n_groups;
  constexpr int kChunkElems = 16 / sizeof(Tin);  // elements per 16-byte copy
  constexpr int kChunksPerRow = kTfVox / kChunkElems;
  int cur_g = -1;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const int g = (int)(t / per_group);
    const int64_t r = t % per_group;
    const int c = (int)(r / vt_count);
    const int64_t v0 = (r % vt_count) * kTfVox;
    const TransformGroup& G = a.g[g];
    __syncthreads();  // the previous tile's reads of Xs (and Tt) are done
    if (GATHER) {
      // source columns and b0 factors of this tile's voxels, then every input row
      for (int vv = tid; vv < kTfVox; vv += blockDim.x) {  // the block may have fewer than 128 threads
        const int64_t v = v0 + vv;
        int64_t src = -1;
        float inv = 0.f;
        if (v < a.n_vox) {
          src = a.index[v];
          if (src < 0 || src >= a.n_src) {
            if (a.err) atomicCAS(a.err, 0, kErrGatherIndex);
            src = -1;
          } else if (a.b0) {
            const float b = a.b0[src];
            inv = b > 0.f ? 1.f / b : 0.f;
          } else {
            inv = 1.f;
          }
        }
        sidx[vv] = src;
        sinv[vv] = inv;
      }
      __syncthreads();
      const Tin* Xg = reinterpret_cast<const Tin*>(a.X) + (G.x_row0 + (int64_t)c * G.x_cstride) * a.ldx;
      for (int i = tid; i < G.n_in * kTfVox; i += blockDim.x) {
        const int j = i / kTfVox, vv = i % kTfVox;
        const int64_t src = sidx[vv];
        reinterpret_cast<float*>(Xs)[i] = src >= 0 ? ldf(Xg + (int64_t)j * a.ldx + src) * sinv[vv] : 0.f;
      }
    } else {
      // input rows of this tile: all copies in flight at once, zero past n_vox
      const Tin* X = reinterpret_cast<const Tin*>(a.X) + (G.x_row0 + (int64_t)c * G.x_cstride) * a.ldx + v0;
      const uint32_t xs_base = (uint32_t)__cvta_generic_to_shared(Xs);
      for (int i = tid; i < G.n_in * kChunksPerRow; i += blockDim.x) {
        const int j = i / kChunksPerRow, ch = i % kChunksPerRow;
        const int64_t vv = v0 + (int64_t)ch * kChunkElems;
        const int64_t left = a.n_vox - vv;
        const int bytes = left >= kChunkElems ? 16 : (left > 0 ? (int)left * (int)sizeof(Tin) : 0);
        const Tin* src = X + (int64_t)j * a.ldx + (int64_t)ch * kChunkElems;
        cp_async16(xs_base + (uint32_t)((j * kTfVox + ch * kChunkElems) * sizeof(Tin)), bytes > 0 ? src : X, bytes);
      }
    }
    if (g != cur_g) {  // the group's operator, transposed: Tt[j][o] = T[o][j], zero past n_out
      for (int i = tid; i < G.n_in * ldt; i += blockDim.x) {
        const int j = i / ldt, o = i % ldt;
        Tt[i] = o < G.n_out ? G.T[(int64_t)o * G.n_in + j] : 0.f;
      }
      cur_g = g;
    }
    cp_async_wait_all();
    __syncthreads();
    if (og * kTfOpt < G.n_out) {
      float acc[kTfOpt][4];
#pragma unroll
      for (int o = 0; o < kTfOpt; ++o)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[o][v] = 0.f;
      const float* tcol = Tt + og * kTfOpt;
      const Ts* xq = Xs + 4 * q;
#pragma unroll 2
      for (int j = 0; j < G.n_in; ++j) {
        const float4 x = ld_x4(xq + j * kTfVox);
        const float4 t0 = *reinterpret_cast<const float4*>(tcol + j * ldt);
        const float4 t1 = *reinterpret_cast<const float4*>(tcol + j * ldt + 4);
        const float4 t2 = *reinterpret_cast<const float4*>(tcol + j * ldt + 8);
        const float tv[kTfOpt] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
#pragma unroll
        for (int o = 0; o < kTfOpt; ++o) {
          acc[o][0] = fmaf(tv[o], x.x, acc[o][0]);
          acc[o][1] = fmaf(tv[o], x.y, acc[o][1]);
          acc[o][2] = fmaf(tv[o], x.z, acc[o][2]);
          acc[o][3] = fmaf(tv[o], x.w, acc[o][3]);
        }
      }
      Tout* Y = reinterpret_cast<Tout*>(a.Y) + (G.y_row0 + (int64_t)c * G.y_cstride + og * kTfOpt) * a.ldy + v0 + 4 * q;
      const int64_t nv = a.n_vox - (v0 + 4 * q);
#pragma unroll
      for (int o = 0; o < kTfOpt; ++o) {
        if (og * kTfOpt + o < G.n_out) {
          Tout* y = Y + (int64_t)o * a.ldy;
          if (nv >= 4) {
            st_y4(y, acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (v < nv) stf(y + v, acc[o][v]);
          }
        }
      }
    }
  }
}

template <typename Tin, typename Tout, bool GATHER = false>
static cudaError_t transform_dispatch(const TransformArgs& a, int n_groups, int max_out, cudaStream_t st) {
  int max_in = 0;
  for (int g = 0; g < n_groups; ++g) max_in = std::max(max_in, a.g[g].n_in);
  if (GATHER && (max_out > kTfMaxOut || max_in > 128)) return cudaErrorInvalidValue;
  if (max_out <= kTfMaxOut && max_in <= 128) {
    const int og_count = (max_out + kTfOpt - 1) / kTfOpt;
    const int threads = 32 * og_count;
    const size_t smem = (size_t)max_in * kTfOpt * og_count * sizeof(float) +
                        (size_t)max_in * kTfVox * (GATHER ? sizeof(float) : sizeof(Tin)) +
                        (GATHER ? (size_t)kTfVox * (sizeof(int64_t) + sizeof(float)) : 0);
    auto kern = transform_staged_kernel<Tin, Tout, GATHER>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.n_vox + kTfVox - 1) / kTfVox * a.channels * n_groups;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(1, per_sm) * sms));
    { kern<<<grid, threads, smem, st>>>(a, n_groups, og_count, max_in); count_launch(); }
    return cudaGetLastError();
  }
  constexpr int VPT = 2;
  const unsigned gx = (unsigned)((a.n_vox + 128 * VPT - 1) / (128 * VPT));
  if (max_out <= 16) {
    const int och = 1;
    dim3 grid(gx, a.channels * och, n_groups);
    { transform_simt_kernel<Tin, Tout, 16, VPT><<<grid, 128, 0, st>>>(a, och); count_launch(); }
  } else {
    const int och = (max_out + 47) / 48;
    dim3 grid(gx, a.channels * och, n_groups);
    { transform_simt_kernel<Tin, Tout, 48, VPT><<<grid, 128, 0, st>>>(a, och); count_launch(); }
  }
  return cudaGetLastError();
}

cudaError_t launch_transform_gather(const TransformArgs& a, int n_groups, int max_out, int in_t, int out_t,
                                    cudaStream_t st) {
  TraceScope trace("signal2sh_gather", st);
  if (a.n_vox == 0) return cudaSuccess;
  if (in_t == 0 && out_t == 0) return transform_dispatch<float, float, true>(a, n_groups, max_out, st);
  if (in_t == 1 && out_t == 0) return transform_dispatch<__nv_bfloat16, float, true>(a, n_groups, max_out, st);
  if (in_t == 0 && out_t == 1) return transform_dispatch<float, __nv_bfloat16, true>(a, n_groups, max_out, st);
  return transform_dispatch<__nv_bfloat16, __nv_bfloat16, true>(a, n_groups, max_out, st);
}

cudaError_t launch_transform_simt(const TransformArgs& a, int n_groups, int max_out, int in_t, int out_t,
                                  cudaStream_t st) {
  TraceScope trace("transform_simt", st);
  if (a.n_vox == 0) return cudaSuccess;
  if (in_t == 0 && out_t == 0) return transform_dispatch<float, float>(a, n_groups, max_out, st);
  if (in_t == 1 && out_t == 0) return transform_dispatch<__nv_bfloat16, float>(a, n_groups, max_out, st);
  if (in_t == 0 && out_t == 1) return transform_dispatch<float, __nv_bfloat16>(a, n_groups, max_out, st);
  return transform_dispatch<__nv_bfloat16, __nv_bfloat16>(a, n_groups, max_out, st);
}

// ---------------------------------------------------------------------------
// Ring-tied kernel weights: one weight for the origin and one per ring, shared by
// the ring's points (kernel point order: origin, ring 1 sectors, ring 2, ...).
//   expand: w[e][k] = w_ring[e][ring(k)],  ring(0) = 0, ring(k) = 1 + (k-1)/sectors
//   reduce: dw_ring[e][r] = sum over the ring's points of dw[e][k]  (the adjoint)
// e runs over the n_e = c_out * S_out * c_in * S_in weight entries.
// ---------------------------------------------------------------------------
__global__ void ring_expand_kernel(const float* __restrict__ w_ring, float* __restrict__ w, int64_t n_e, int K,
                                   int rings, int sectors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_e * K) return;
  const int64_t e = i / K;
  const int k = (int)(i % K);
  const int r = k == 0 ? 0 : 1 + (k - 1) / sectors;
  w[i] = w_ring[e * (rings + 1) + r];
}

__global__ void ring_reduce_kernel(const float* __restrict__ dw, float* __restrict__ dw_ring, int64_t n_e, int K,
                                   int rings, int sectors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_e * (rings + 1)) return;
  const int64_t e = i / (rings + 1);
  const int r = (int)(i % (rings + 1));
  const float* src = dw + e * K;
  float acc = 0.f;
  if (r == 0) {
    acc = src[0];
  } else {
    for (int q = 0; q < sectors; ++q) acc += src[1 + (r - 1) * sectors + q];  // fixed order
  }
  dw_ring[i] = acc;
}

cudaError_t launch_ring_weights(const float* src, float* dst, int64_t n_e, int K, int rings, int sectors, bool expand,
                                cudaStream_t st) {
  TraceScope trace(expand ? "lsc_ring_expand" : "lsc_ring_reduce", st);
  const int64_t n = n_e * (expand ? K : rings + 1);
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (expand) {
    ring_expand_kernel<<<grid, 256, 0, st>>>(src, dst, n_e, K, rings, sectors);
  } else {
    ring_reduce_kernel<<<grid, 256, 0, st>>>(src, dst, n_e, K, rings, sectors);
  }
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Collapsed LSC operator.  For every shell pair (s, s') in the window
//   W[(s,co,a)][(s',ci,b)] = sum_k w[co,s,ci,s',k] M_{s,s'}[k][a][b] (M_{s,s'} = M_s in the resampled form)
// a small GEMM per shell pair: [channel pairs x K] x [K x (a,b)].  One block: 64
// consecutive channel pairs p = co c_in + ci of one shell pair x 256 consecutive (a, b)
// entries; K in chunks of 56 kernel points (one chunk for K <= 56), M_{s,s'}[k][ab0 ..
// ab0+255] and w[p][k] staged in shared memory.  Warp = 8 pairs, lane = 8 consecutive
// entries: per kernel point two broadcast and two 128-bit shared loads feed 64 FMAs.
// The finished block goes back through shared memory and is written to W, a warp per
// run of a row (s, co, a): the block's channels ci and their b entries, contiguous in W;
// and to Wt (runs along a).  Shell pairs outside the window write zeros.
// ---------------------------------------------------------------------------
constexpr int kBwP = 64, kBwAB = 128, kBwKC = 56;  // pairs, (a,b) entries, kernel points per chunk
constexpr size_t kBwSmem = sizeof(float) * kBwKC * (kBwAB + kBwP);  // a chunk (M + w); then the results
static_assert(kBwP * kBwAB <= kBwKC * (kBwAB + kBwP), "the results fit a staged chunk's space");

template <typename TW>
__global__ void __launch_bounds__(256, 3) build_w_kernel(const __grid_constant__ LscDims d, const float* __restrict__ w,
                                                      const float* __restrict__ M, TW* __restrict__ W,
                                                      TW* __restrict__ Wt) {
  extern __shared__ float4 blk4[];  // chunk: ms [kBwKC][kBwAB], ws [kBwKC][kBwP]; then results [kBwP][kBwAB]
  float* blk = reinterpret_cast<float*>(blk4);
  float* ms = blk;
  float* ws = blk + kBwKC * kBwAB;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int pair = blockIdx.y;  // s * s_in + s'
  const int s = pair / d.s_in, sp = pair % d.s_in;
  const bool in_win = sp >= d.win_lo[s] && sp < d.win_hi[s];
  const int nab = d.n_out * d.n_in, npairs = d.c_out * d.c_in;
  const int p0 = blockIdx.x * kBwP;
  const int np = min(kBwP, npairs - p0);
  const int ab0 = blockIdx.z * kBwAB, nabc = min(kBwAB, nab - ab0);  // this block's (a,b) range
  // acc[i][e2] = entries 2 e2, 2 e2 + 1 of pair i: packed FP32x2 FMAs (each lane rounds as fmaf)
  float2 acc[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int e = 0; e < 2; ++e) acc[i][e] = make_float2(0.f, 0.f);
  if (in_win) {
    const float* Ms = M + s * d.m_stride_s + sp * d.m_stride_sp + ab0;
    for (int k0 = 0; k0 < d.K; k0 += kBwKC) {
      const int kc = min(kBwKC, d.K - k0);
      __syncthreads();  // the previous chunk is consumed
      // M rows k0 .. k0 + kc - 1: thread tid loads entry tid of each (zero past the ranges)
#pragma unroll 8
      for (int i = tid; i < kBwKC * kBwAB; i += 256) {
        const int kk = i / kBwAB, t = i % kBwAB;
        ms[i] = (kk < kc && t < nabc) ? __ldg(Ms + (int64_t)(k0 + kk) * nab + t) : 0.f;
      }
      // w[p][k0 + kk] for the block's pairs, pair index fastest (conflict-free stores)
#pragma unroll
      for (int e = 0; e < kBwKC * kBwP / 256; ++e) {
        const int idx = tid + 256 * e, pp = idx % kBwP, kk = idx / kBwP, pr = p0 + pp;
        float v = 0.f;
        if (pp < np && kk < kc) {
          const int co = pr / d.c_in, ci = pr - co * d.c_in;
          v = __ldg(w + ((((int64_t)co * d.s_out + s) * d.c_in + ci) * d.s_in + sp) * d.K + k0 + kk);
        }
        ws[kk * kBwP + pp] = v;
      }
      __syncthreads();
      const float4* ms4 = reinterpret_cast<const float4*>(ms) + lane;
      const float4* ws4 = reinterpret_cast<const float4*>(ws) + 2 * warp;
#pragma unroll 2
      for (int kk = 0; kk < kc; ++kk) {
        const float4 m0 = ms4[kk * (kBwAB / 4)];
        const float4 w0 = ws4[kk * (kBwP / 4)], w1 = ws4[kk * (kBwP / 4) + 1];
        const float2 mv[2] = {make_float2(m0.x, m0.y), make_float2(m0.z, m0.w)};
        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 wi = make_float2(wv[i], wv[i]);
#pragma unroll
          for (int e = 0; e < 2; ++e) acc[i][e] = __ffma2_rn(wi, mv[e], acc[i][e]);
        }
      }
    }
  }
  __syncthreads();
  // results [p][t]: pair p = 8 warp + i, entry t = 8 lane + e
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    blk4[(8 * warp + i) * (kBwAB / 4) + lane] = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
  }
  __syncthreads();
  // Stores: one warp per output run (a pair's row segment), lanes along the contiguous index
  const int a_lo = ab0 / d.n_in, a_hi = (ab0 + nabc - 1) / d.n_in;  // a range touched by this chunk
  const int na = a_hi - a_lo + 1;
  const int b_lo = na > 1 ? 0 : ab0 % d.n_in, b_hi = na > 1 ? d.n_in - 1 : (ab0 + nabc - 1) % d.n_in;
  const int nb = b_hi - b_lo + 1;
  // W: for each output channel co of the block's pairs and each a of the chunk, the block's
  // channels ci with their b entries form one run of W's row (s, co, a) (columns s' in_blk
  // + ci n_in + b, contiguous over (ci, b)); a warp per run, lanes along the run, the lane's
  // (ci, b) advanced incrementally
  const int co_lo = p0 / d.c_in, nco = (p0 + np - 1) / d.c_in - co_lo + 1;
  for (int r = warp; r < nco * na; r += 8) {
    const int ko = r / na, ai = r - ko * na, co = co_lo + ko, aa = a_lo + ai;
    const int ci0 = max(0, p0 - co * d.c_in), ci1 = min(d.c_in, p0 + np - co * d.c_in);
    const int b0 = max(0, ab0 - aa * d.n_in), b1 = min(d.n_in, ab0 + nabc - aa * d.n_in);
    const int len = (ci1 - ci0) * d.n_in;
    TW* dst = W + (((int64_t)s * d.c_out + co) * d.n_out + aa) * d.ldW + (int64_t)sp * d.in_blk + (int64_t)ci0 * d.n_in;
    const int src0 = (co * d.c_in + ci0 - p0) * kBwAB + aa * d.n_in - ab0;  // + (ci - ci0) kBwAB + b
    int cj = lane / d.n_in, bj = lane - cj * d.n_in;
    for (int j = lane; j < len; j += 32) {
      if (bj >= b0 && bj < b1) stf(dst + j, blk[src0 + cj * kBwAB + bj]);
      bj += 32;
      while (bj >= d.n_in) {
        bj -= d.n_in;
        ++cj;
      }
    }
  }
  if (!Wt) return;
  // Wt: row (s', ci, b), columns s*out_blk + co*n_out + a; run r = (pair, b)
  for (int r = warp; r < np * nb; r += 8) {
    const int p = r / nb, bi = r - p * nb, pr = p0 + p, co = pr / d.c_in, ci = pr - co * d.c_in, bb = b_lo + bi;
    const float* src = blk + p * kBwAB;
    TW* dst = Wt + (((int64_t)sp * d.c_in + ci) * d.n_in + bb) * d.ldWt + (int64_t)s * d.out_blk + (int64_t)co * d.n_out;
    for (int aa = a_lo + lane; aa <= a_hi; aa += 32) {
      const int t = aa * d.n_in + bb;
      if (t >= ab0 && t < ab0 + nabc) stf(dst + aa, src[t - ab0]);
    }
  }
}

__global__ void build_bias_kernel(const __grid_constant__ LscDims d, const float* __restrict__ b,
                                  const float* __restrict__ q, float* __restrict__ bias_vec) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.rows_out) return;
  const int per_out = d.c_out * d.n_out;
  const int s = (int)(r / per_out), co = (int)((r / d.n_out) % d.c_out), aa = (int)(r % d.n_out);
  bias_vec[r] = b ? b[co * d.s_out + s] * q[s * d.n_out + aa] : 0.f;
}

cudaError_t launch_build_w(const LscDims& d, const float* w, const float* b, const float* M, const float* q,
                           void* W, void* Wt, float* bias_vec, int w_t, cudaStream_t st) {
  TraceScope trace("lsc_build_w", st);
  const size_t es = w_t == 0 ? 4 : 2;
  const int nab = d.n_out * d.n_in, npairs = d.c_out * d.c_in;
  cudaError_t e;
  // padding columns between shell blocks stay zero
  if (d.in_blk != (int64_t)d.c_in * d.n_in) {
    e = cudaMemsetAsync(W, 0, (size_t)d.rows_out * d.ldW * es, st);
    if (e != cudaSuccess) return e;
  }
  if (Wt && d.out_blk != (int64_t)d.c_out * d.n_out) {
    e = cudaMemsetAsync(Wt, 0, (size_t)d.rows_in * d.ldWt * es, st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((npairs + kBwP - 1) / kBwP), (unsigned)(d.s_out * d.s_in),
            (unsigned)((nab + kBwAB - 1) / kBwAB));
  const size_t smem = kBwSmem;
  if (w_t == 0) {
    e = cudaFuncSetAttribute(build_w_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    { build_w_kernel<float><<<grid, 256, smem, st>>>(d, w, M, (float*)W, (float*)Wt); count_launch(); }
  } else {
    e = cudaFuncSetAttribute(build_w_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    { build_w_kernel<__nv_bfloat16><<<grid, 256, smem, st>>>(d, w, M, (__nv_bfloat16*)W, (__nv_bfloat16*)Wt); count_launch(); }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || !bias_vec) return e;
  return launch_build_bias(d, b, q, bias_vec, st);
}

cudaError_t launch_build_bias(const LscDims& d, const float* b, const float* q, float* bias_vec, cudaStream_t st) {
  { build_bias_kernel<<<(unsigned)((d.rows_out + 255) / 256), 256, 0, st>>>(d, b, q, bias_vec); count_launch(); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row GEMM over voxels (LSC forward and input gradient), 128 x 128 x 8 tiles,
// 256 threads, 8 x 8 outputs per thread.
// ---------------------------------------------------------------------------
template <typename TA, typename TX>
__global__ void __launch_bounds__(256) row_gemm_simt_kernel(const __grid_constant__ RowGemmArgs p) {
  constexpr int BM = 128, BN = 128, BK = 8;
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Xs[BK][BN];
  const RowGemmGroup& g = p.g[blockIdx.z];
  const int m0 = blockIdx.y * BM;
  if (m0 >= g.R) return;
  const int64_t v0 = (int64_t)blockIdx.x * BN;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const TA* At = reinterpret_cast<const TA*>(p.At);
  const TX* X = reinterpret_cast<const TX*>(p.X);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int lk = t / 32, lc = (t % 32) * 4;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    float ra[4], rx[4];
    const int k = k0 + lk;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + lc + i;
      ra[i] = (k < g.K && r < g.R) ? ldf(At + (g.at_row0 + k) * p.ldat + g.at_col0 + r) : 0.f;
      const int64_t vv = v0 + lc + i;
      rx[i] = (k < g.K && vv < p.n_vox) ? ldf(X + (g.x_row0 + k) * p.ldx + vv) : 0.f;
    }
    __syncthreads();
    *reinterpret_cast<float4*>(&As[lk][lc]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
    *reinterpret_cast<float4*>(&Xs[lk][lc]) = make_float4(rx[0], rx[1], rx[2], rx[3]);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[kk][tx * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float xv8[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], xv8[j], acc[i][j]);
    }
  }
  TX* Y = reinterpret_cast<TX*>(p.Y);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (r >= g.R) continue;
    const float bias = p.bias ? p.bias[g.y_row0 + r] : 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t vv = v0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (vv < p.n_vox) stf(Y + (g.y_row0 + r) * p.ldy + vv, acc[i][j] + bias);
    }
  }
}

cudaError_t launch_row_gemm_simt(const RowGemmArgs& a, int n_groups, int max_R, int act_t, cudaStream_t st) {
  TraceScope trace("lsc_gemm_simt", st);
  if (a.n_vox == 0) return cudaSuccess;
  dim3 grid((unsigned)((a.n_vox + 127) / 128), (unsigned)((max_R + 127) / 128), n_groups);
  if (act_t == 0)
    { row_gemm_simt_kernel<float, float><<<grid, 256, 0, st>>>(a); count_launch(); }
  else
    { row_gemm_simt_kernel<__nv_bfloat16, __nv_bfloat16><<<grid, 256, 0, st>>>(a); count_launch(); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weight-gradient GEMM: reduction over a voxel split, 128 x 128 tiles, BK = 16
// voxels.  Column N of every group is the virtual all-ones input row, so the
// same pass yields the row sums of dY needed for the bias gradient.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) wgrad_simt_kernel(const __grid_constant__ WgradArgs p, int mtiles) {
  constexpr int BM = 128, BN = 128, BK = 16;
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int gi = blockIdx.y / mtiles, mt = blockIdx.y % mtiles;
  const WgradGroup& g = p.g[gi];
  const int m0 = mt * BM, n0 = blockIdx.x * BN;
  const int Ne = g.N + 1;  // + ones column
  if (m0 >= g.M || n0 >= Ne) return;
  const int64_t vs = (int64_t)blockIdx.z * p.vox_per_split;
  const int64_t ve = min(p.n_vox, vs + p.vox_per_split);
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const T* dY = reinterpret_cast<const T*>(p.dY);
  const T* X = reinterpret_cast<const T*>(p.X);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int lr = t / 2, lv = (t % 2) * 8;
  for (int64_t k0 = vs; k0 < ve; k0 += BK) {
    float ra[8], rb[8];
    const int m = m0 + lr, n = n0 + lr;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t vv = k0 + lv + i;
      const bool in = vv < ve;
      ra[i] = (in && m < g.M) ? ldf(dY + (g.m_row0 + m) * p.lddy + vv) : 0.f;
      rb[i] = (in && n < g.N) ? ldf(X + (g.x_row0 + n) * p.ldx + vv) : ((in && n == g.N) ? 1.f : 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      As[lv + i][lr] = ra[i];
      Bs[lv + i][lr] = rb[i];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }
  float* P = p.P + (int64_t)blockIdx.z * p.split_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (n > g.N) continue;
      const int64_t col = (n == g.N) ? p.ones_col : g.n_col0 + n;
      P[(g.m_row0 + m) * p.ldp + col] = acc[i][j];
    }
  }
}

cudaError_t launch_wgrad_simt(const WgradArgs& a, int n_groups, int max_M, int max_N, int splits, int act_t,
                              cudaStream_t st) {
  TraceScope trace("lsc_wgrad_simt", st);
  const int mtiles = (max_M + 127) / 128;
  dim3 grid((unsigned)((max_N + 1 + 127) / 128), (unsigned)(mtiles * n_groups), (unsigned)splits);
  if (act_t == 0)
    { wgrad_simt_kernel<float><<<grid, 256, 0, st>>>(a, mtiles); count_launch(); }
  else
    { wgrad_simt_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(a, mtiles); count_launch(); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dW -> dw (kernel-point weights) and db.  For a windowed shell pair,
//   dw[co,s,ci,s',k] = sum_{a,b} M_{s,s'}[k][a][b] G[(s,co,a)][(s',ci,b)],  G = sum_split P;
// a block owns 32 channel pairs x all K and walks (a,b) in chunks of 128.
// ---------------------------------------------------------------------------
constexpr int kDwAbPart = 256;  // (a,b) entries per partial sum

// Partials stored row-major (p_cs = 1; the CUDA-core weight gradient).
__global__ void __launch_bounds__(256) reduce_dw_kernel(const __grid_constant__ LscDims d, const float* __restrict__ P,
                                                        int64_t p_rs, int64_t p_cs, int64_t split_stride, int splits,
                                                        const float* __restrict__ M, float* __restrict__ dwp,
                                                        int64_t part_stride) {
  // block: 64 channel pairs x 64 kernel points x one (a,b) part; thread: 4 pairs x 4 points;
  // the part is walked in chunks of 32.  Writes partial sums dwp[part][dw index].
  constexpr int PT = 64, KT = 64, AB = 32;
  __shared__ __align__(16) float gs[AB][PT + 4];
  __shared__ __align__(16) float ms_[AB][KT + 4];
  const int npairs = d.c_out * d.c_in, nab = d.n_out * d.n_in;
  const int nparts = (nab + kDwAbPart - 1) / kDwAbPart;
  const int pair = blockIdx.z / nparts, part = blockIdx.z % nparts;
  const int s = pair / d.s_in, sp = pair % d.s_in;
  const int p0 = blockIdx.y * PT, k0 = blockIdx.x * KT;
  const bool in_win = sp >= d.win_lo[s] && sp < d.win_hi[s];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int ab_end = min(nab, (part + 1) * kDwAbPart);
  float acc[4][4] = {};
  if (in_win) {
    // software pipeline: the next chunk's loads are issued before this chunk's FMAs and
    // summed after them (up to four splits held raw in registers)
    constexpr int kRaw = 4;
    float raw[8][kRaw], mv_n[8];
    auto issue = [&](int ab0) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int idx = threadIdx.x + 256 * e;
        {
          const int t = idx % AB, pp = idx / AB, pr = p0 + pp, ab = ab0 + t;
#pragma unroll
          for (int z = 0; z < kRaw; ++z) raw[e][z] = 0.f;
          if (pr < npairs && ab < ab_end) {
            const int co = pr / d.c_in, ci = pr % d.c_in;
            const int aa = ab / d.n_in, bb = ab % d.n_in;
            const int64_t off = (((int64_t)s * d.c_out + co) * d.n_out + aa) * p_rs +
                                (((int64_t)sp * d.c_in + ci) * d.n_in + bb) * p_cs;
#pragma unroll
            for (int z = 0; z < kRaw; ++z)
              if (z < splits) raw[e][z] = P[z * split_stride + off];
            for (int z = kRaw; z < splits; ++z) raw[e][kRaw - 1] += P[z * split_stride + off];
          }
        }
        {
          const int t = idx % AB, kk = idx / AB, ab = ab0 + t, k = k0 + kk;
          mv_n[e] = (ab < ab_end && k < d.K) ? M[s * d.m_stride_s + sp * d.m_stride_sp + (int64_t)k * nab + ab] : 0.f;
        }
      }
    };
    auto stage = [&]() {  // summed values of the issued chunk into shared memory
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int idx = threadIdx.x + 256 * e;
        float v = raw[e][0];
#pragma unroll
        for (int z = 1; z < kRaw; ++z) v += raw[e][z];
        gs[idx % AB][idx / AB] = v;
        ms_[idx % AB][idx / AB] = mv_n[e];
      }
    };
    issue(part * kDwAbPart);
    for (int ab0 = part * kDwAbPart; ab0 < ab_end; ab0 += AB) {
      __syncthreads();  // the previous chunk's FMAs are done with gs / ms_
      stage();
      __syncthreads();
      if (ab0 + AB < ab_end) issue(ab0 + AB);
      const int nt = min(AB, ab_end - ab0);
      for (int t = 0; t < nt; ++t) {
        const float4 g4 = *reinterpret_cast<const float4*>(&gs[t][ty * 4]);
        const float4 m4 = *reinterpret_cast<const float4*>(&ms_[t][tx * 4]);
        const float gv[4] = {g4.x, g4.y, g4.z, g4.w}, mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(gv[i], mv[j], acc[i][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pr = p0 + ty * 4 + i;
    if (pr >= npairs) continue;
    const int co = pr / d.c_in, ci = pr % d.c_in;
    float* out = dwp + part * part_stride + ((((int64_t)co * d.s_out + s) * d.c_in + ci) * d.s_in + sp) * d.K;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tx * 4 + j;
      if (k < d.K) out[k] = in_win ? acc[i][j] : 0.f;
    }
  }
}

// Partials stored transposed (p_rs = 1: P's rows (s, co, a) are contiguous, a fastest; the
// tensor-core weight gradient).  One block: 64 channel pairs x 56 kernel points x one part
// of kDwAbPart (a,b) entries, walked with a fastest (ab = b n_out + a: the order of P's
// rows and of Mt, per kernel point [b][a]) in chunks of 32, the next chunk's loads in
// flight during the current one's FMAs.  Staged per chunk: G = the sum of P's splits, as
// gs[entry][pair], and Mt as ms_[entry][slot] with kernel point k = 7 kg + j in slot
// 8 kg + j (slot 8 kg + 7 zero).  A loading thread covers 4 consecutive pairs (or slots)
// at 2 entries: half-warps run along a in global memory, one 128-bit shared store each.
// Four warp-aligned teams of 64 threads take every fourth entry; a thread accumulates
// pairs 4 pg + {0..3}, 32 + 4 pg + {0..3} x points 7 kg + {0..6} (four conflict-free 128-bit
// shared loads per 56 FMAs); the teams' sums meet in shared memory at the end.
constexpr int kDtP = 64, kDtK = 56, kDtSlots = 64, kDtAB = 32, kDtTeams = 4, kDtRaw = 3;
static_assert(kDwAbPart % kDtAB == 0, "whole chunks per part");

__global__ void __launch_bounds__(256) reduce_dw_t_kernel(const __grid_constant__ LscDims d, const float* __restrict__ P,
                                                          int64_t p_cs, int64_t split_stride, int splits,
                                                          const float* __restrict__ Mt, float* __restrict__ dwp,
                                                          int64_t part_stride) {
  __shared__ __align__(16) float gs[kDtAB][kDtP + 4];
  __shared__ __align__(16) float ms_[kDtAB][kDtSlots + 4];
  __shared__ __align__(16) float red[kDtP * kDtK];
  __shared__ int64_t base_p[kDtP];  // P offset of (pair, a = 0, b = 0)
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int npairs = d.c_out * d.c_in, nab = d.n_out * d.n_in;
  const int nparts = (nab + kDwAbPart - 1) / kDwAbPart;
  const int pair = blockIdx.z / nparts, part = blockIdx.z % nparts;
  const int s = pair / d.s_in, sp = pair % d.s_in;
  const int p0 = blockIdx.y * kDtP, k0 = blockIdx.x * kDtK;
  const int np = min(kDtP, npairs - p0);
  const bool in_win = sp >= d.win_lo[s] && sp < d.win_hi[s];
  const int ab_beg = part * kDwAbPart, ab_end = min(nab, ab_beg + kDwAbPart);
  // compute roles
  const int team = warp / 2, t64 = tid % 64, pg = t64 % 8, kg = t64 / 8;
  // load roles: quad q (pairs or slots 4q .. 4q+3), entries tl and tl + 16
  const int q = 2 * warp + lane / 16, tl = lane % 16;
  float acc[8][7];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 7; ++j) acc[i][j] = 0.f;
  if (in_win) {
    if (tid < kDtP) {
      const int pr = p0 + tid, co = pr / d.c_in, ci = pr - co * d.c_in;
      base_p[tid] = tid < np ? ((int64_t)s * d.c_out + co) * d.n_out + ((int64_t)sp * d.c_in + ci) * d.n_in * p_cs : 0;
    }
    __syncthreads();
    const float* Ms = Mt + s * d.m_stride_s + sp * d.m_stride_sp;
    // this thread's kernel points of slot quad q (slot 8 kg + j holds k = 7 kg + j, j < 7)
    int kq[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int slot = 4 * q + c, j = slot % 8;
      kq[c] = j < 7 ? k0 + 7 * (slot / 8) + j : -1;
    }
    float raw[2][4][kDtRaw], mv[2][4];
    auto issue = [&](int ab0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ab = ab0 + tl + 16 * h;
        const bool ok = ab < ab_end;
        const int bb = ok ? ab / d.n_out : 0, aa = ok ? ab - bb * d.n_out : 0;
        const int64_t off = aa + (int64_t)bb * p_cs;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int pp = 4 * q + c;
          const bool on = ok && pp < np;
          const float* src = P + (on ? base_p[pp] + off : 0);
#pragma unroll
          for (int z = 0; z < kDtRaw; ++z) raw[h][c][z] = (on && z < splits) ? __ldg(src + z * split_stride) : 0.f;
          for (int z = kDtRaw; z < splits; ++z) raw[h][c][kDtRaw - 1] += on ? __ldg(src + z * split_stride) : 0.f;
          const int k = kq[c];
          mv[h][c] = (ok && k >= 0 && k < d.K) ? __ldg(Ms + (int64_t)k * nab + ab) : 0.f;
        }
      }
    };
    issue(ab_beg);
    for (int ab0 = ab_beg; ab0 < ab_end; ab0 += kDtAB) {
      __syncthreads();  // the previous chunk's FMAs are done with gs / ms_
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float g[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          g[c] = raw[h][c][0];
#pragma unroll
          for (int z = 1; z < kDtRaw; ++z) g[c] += raw[h][c][z];
        }
        *reinterpret_cast<float4*>(&gs[tl + 16 * h][4 * q]) = make_float4(g[0], g[1], g[2], g[3]);
        *reinterpret_cast<float4*>(&ms_[tl + 16 * h][4 * q]) = make_float4(mv[h][0], mv[h][1], mv[h][2], mv[h][3]);
      }
      __syncthreads();
      if (ab0 + kDtAB < ab_end) issue(ab0 + kDtAB);
      // entries past the part's end were staged as zeros: a fixed trip count
#pragma unroll
      for (int u = 0; u < kDtAB / kDtTeams; ++u) {
        const int t = team + kDtTeams * u;
        const float4 g0 = *reinterpret_cast<const float4*>(&gs[t][4 * pg]);
        const float4 g1 = *reinterpret_cast<const float4*>(&gs[t][32 + 4 * pg]);
        const float4 m0 = *reinterpret_cast<const float4*>(&ms_[t][8 * kg]);
        const float4 m1 = *reinterpret_cast<const float4*>(&ms_[t][8 * kg + 4]);
        const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        const float mm[7] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 7; ++j) acc[i][j] = fmaf(gv[i], mm[j], acc[i][j]);
      }
    }
    // the teams' sums, in team order (deterministic); thread (pg, kg) owns pairs
    // 4 pg + i (i < 4) and 32 + 4 pg + i - 4 (i >= 4), points 7 kg + j
    auto ridx = [&](int i, int j) { return ((i < 4 ? 4 * pg + i : 28 + 4 * pg + i)) * kDtK + 7 * kg + j; };
    for (int tm = 1; tm < kDtTeams; ++tm) {
      __syncthreads();
      if (team == tm) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 7; ++j) {
            float& x = red[ridx(i, j)];
            x = tm == 1 ? acc[i][j] : x + acc[i][j];
          }
      }
    }
    __syncthreads();
    if (team == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 7; ++j) acc[i][j] += red[ridx(i, j)];
    }
  }
  if (team != 0) return;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int pr = p0 + (i < 4 ? 4 * pg + i : 28 + 4 * pg + i);
    if (pr >= npairs) continue;
    const int co = pr / d.c_in, ci = pr - co * d.c_in;
    float* out = dwp + part * part_stride + ((((int64_t)co * d.s_out + s) * d.c_in + ci) * d.s_in + sp) * d.K;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const int k = k0 + 7 * kg + j;
      if (k < d.K) out[k] = acc[i][j];
    }
  }
}

// dw[i] = sum over parts in order (deterministic)
__global__ void sum_parts_kernel(const float* __restrict__ dwp, int64_t part_stride, int nparts, int64_t n,
                                 float* __restrict__ dw) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int p = 0; p < nparts; ++p) a += dwp[p * part_stride + i];
    dw[i] = a;
  }
}

__global__ void reduce_db_kernel(const __grid_constant__ LscDims d, const float* __restrict__ P, int64_t p_rs,
                                 int64_t p_cs, int64_t split_stride, int splits, int64_t ones_col,
                                 const float* __restrict__ q, float* __restrict__ db) {
  const int co = blockIdx.x, s = blockIdx.y;
  const int64_t row0 = ((int64_t)s * d.c_out + co) * d.n_out;
  float acc = 0.f;
  for (int aa = threadIdx.x; aa < d.n_out; aa += 32) {
    float r = 0.f;
    for (int z = 0; z < splits; ++z) r += P[z * split_stride + (row0 + aa) * p_rs + ones_col * p_cs];
    acc = fmaf(q[s * d.n_out + aa], r, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) db[co * d.s_out + s] = acc;
}

size_t reduce_dw_scratch_floats(const LscDims& d) {
  const int nparts = (d.n_out * d.n_in + kDwAbPart - 1) / kDwAbPart;
  return (size_t)nparts * d.c_out * d.s_out * d.c_in * d.s_in * d.K;
}

cudaError_t launch_reduce_dw(const LscDims& d, const float* P, int64_t p_rs, int64_t p_cs, int64_t split_stride,
                             int splits, const float* M, const float* Mt, const float* q, float* dw, float* db,
                             float* scratch, cudaStream_t st) {
  TraceScope trace("lsc_reduce_dw", st);
  if (dw) {
    const int nparts = (d.n_out * d.n_in + kDwAbPart - 1) / kDwAbPart;
    const int64_t n = (int64_t)d.c_out * d.s_out * d.c_in * d.s_in * d.K;
    if (p_rs == 1) {
      dim3 grid((unsigned)((d.K + kDtK - 1) / kDtK), (unsigned)((d.c_out * d.c_in + kDtP - 1) / kDtP),
                (unsigned)(d.s_out * d.s_in * nparts));
      reduce_dw_t_kernel<<<grid, 256, 0, st>>>(d, P, p_cs, split_stride, splits, Mt, scratch, n);
    } else {
      dim3 grid((unsigned)((d.K + 63) / 64), (unsigned)((d.c_out * d.c_in + 63) / 64),
                (unsigned)(d.s_out * d.s_in * nparts));
      reduce_dw_kernel<<<grid, 256, 0, st>>>(d, P, p_rs, p_cs, split_stride, splits, M, scratch, n);
    }
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)std::min<int64_t>(4096, (n + 255) / 256);
    { sum_parts_kernel<<<g, 256, 0, st>>>(scratch, n, nparts, n, dw); count_launch(); }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (db) {
    { reduce_db_kernel<<<dim3(d.c_out, d.s_out), 32, 0, st>>>(d, P, p_rs, p_cs, split_stride, splits, d.rows_in, q, db); count_launch(); }
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace delimit
