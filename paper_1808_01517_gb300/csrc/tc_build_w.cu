// The collapsed LSC operator on the tensor cores (Sec. 2.3, the exact collapse of the
// resample / product / projection steps into one matrix per shell pair):
//   W[(s,co,a)][(s',ci,b)] = sum_k w[co,s,ci,s',k] M_{s,s'}[k][a][b]
// per shell pair a GEMM [channel pairs p = co c_in + ci] x [kernel points k < K] x
// [(a,b) entries], with K <= 64 (padded with zeros to 64).  FP32 operands on the BF16
// tensor cores as three-part splits (x = x0 + x1 + x2 to 2^-27 |x|, the six part
// products down to 2^-18 of the leading one, FP32 accumulation in TMEM): FP32-level
// accuracy before the result is rounded to BF16 (the same rounding point as the
// CUDA-core build).  The parts of M are made once per geometry (M is fixed).
//
// One CTA per (shell pair, 128 channel pairs, 256 (a,b) entries), c_in dividing 128 so
// that a tile holds whole output channels:
//   - the CTA splits its 128 x 64 slice of w into three BF16 parts, written straight into
//     the K-major 128-byte-swizzled operand layout; one thread loads the three M parts
//     (MN-major, four 64-entry atoms x 64 k each) by TMA, issues the 24 MMAs (M = 128,
//     N = 256, K = 16) and commits;
//   - 32 warps read the accumulator (eight per TMEM lane quarter), round to BF16 and
//     scatter it into a staging tile in W's own order [co][a][ci][b] (in the freed
//     operand space), so that every row run of W the tile covers, (s, co, a) with the
//     tile's channels ci and their b entries, is contiguous there;
//   - the warps copy the runs out, 16 bytes per lane where the run is whole and aligned.
// Shell pairs outside the window write zeros.  Every wait is bounded.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace delimit {

namespace {

constexpr int kBwTP = 128;                              // channel pairs per tile (MMA M)
constexpr int kBwTN = 256;                              // (a,b) entries per tile (MMA N)
constexpr int kBwK = 64;                                // kernel points, zero-padded
constexpr uint32_t kBwABytes = kBwTP * kBwK * 2;         // one w part tile: 16 KiB
constexpr uint32_t kBwBBytes = kBwTN * kBwK * 2;         // one M part tile: 4 atoms x 8 KiB
constexpr uint32_t kBwOpBytes = 3 * (kBwABytes + kBwBBytes);  // 144 KiB
constexpr int kBwThreads = 1024;
constexpr int kErrBwLoad = 0x4A00, kErrBwMma = 0x4B00;

// the six part products, largest first: term t multiplies part pa(t) of w with part pb(t) of M
__host__ __device__ constexpr int bw_part_a(int t) { return t == 2 || t == 3 ? 1 : (t == 5 ? 2 : 0); }
__host__ __device__ constexpr int bw_part_b(int t) { return t == 1 || t == 3 ? 1 : (t == 4 ? 2 : 0); }

// two BF16 values' bits in one word, lo in the low half
__device__ __forceinline__ uint32_t bf16_bits2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// (a,b) rows a tile of 256 entries touches, at most
__host__ __device__ constexpr int bw_max_rows(int n_in) { return (kBwTN - 1) / n_in + 2; }

// M_{s,s'} -> its three BF16 parts, per shell pair pg a [64][ldm] MN-major block (kernel
// point k, entry ab; zero past K points and nab entries).  Scalar loads: M's rows of
// n_out n_in floats need not be 16-byte aligned.
__global__ void split_m_kernel(const __grid_constant__ LscDims d, const float* __restrict__ M,
                               __nv_bfloat16* __restrict__ mp, int ldm, int npg) {
  const int64_t n = (int64_t)npg * kBwK * ldm;
  const int nab = d.n_out * d.n_in;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int ab = (int)(i % ldm);
    const int64_t r = i / ldm;
    const int k = (int)(r % kBwK), pg = (int)(r / kBwK);
    const int s = pg / d.s_in, sp = pg - s * d.s_in;
    const float x = (k < d.K && ab < nab) ? M[s * d.m_stride_s + sp * d.m_stride_sp + (int64_t)k * nab + ab] : 0.f;
    const __nv_bfloat16 x0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(x0);
    const __nv_bfloat16 x1 = __float2bfloat16_rn(r1);
    mp[i] = x0;
    mp[n + i] = x1;
    mp[2 * n + i] = __float2bfloat16_rn(r1 - __bfloat162float(x1));
  }
}

}  // namespace

struct BwMaps {
  CUtensorMap b;  // M parts: 2-D {ldm entries, 3 npg 64 rows}, box {64, 64}
};

__global__ void __launch_bounds__(kBwThreads, 1)
    build_w_tc_kernel(const __grid_constant__ BwMaps maps, const __grid_constant__ LscDims d,
                      const float* __restrict__ w, __nv_bfloat16* __restrict__ W, int vec, int* err) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t a_base = sbase, b_base = sbase + 3 * kBwABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kBwOpBytes);  // full, done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t full_bar = smem_u32(bars), done_bar = smem_u32(bars + 1);
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem);  // [nco][na][c_in][n_in] after the MMAs
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int pg = blockIdx.z, s = pg / d.s_in, sp = pg - s * d.s_in;
  const bool in_win = sp >= d.win_lo[s] && sp < d.win_hi[s];
  const int nab = d.n_out * d.n_in, npairs = d.c_out * d.c_in;
  const int p0 = blockIdx.y * kBwTP, np = min(kBwTP, npairs - p0);
  const int ab0 = blockIdx.x * kBwTN, nabc = min(kBwTN, nab - ab0);
  const int npg = d.s_out * d.s_in;
  // c_in divides 128: the tile holds channels co_lo .. co_lo + nco - 1 whole
  const int co_lo = p0 / d.c_in, nco = np / d.c_in;
  const int a_lo = ab0 / d.n_in, na = (ab0 + nabc - 1) / d.n_in - a_lo + 1;
  const int rowlen = d.c_in * d.n_in;
  bool ok = true;
  if (in_win) {
    if (tid == 0) {
      mbar_init(full_bar, 1);
      mbar_init(done_bar, 1);
      *abort_flag = 0;
      fence_mbar_init();
      // the three parts of M (kernel points 0 .. 63 of entries ab0 .., four 64-entry atoms
      // each), in flight while the threads split w
      mbar_arrive_expect_tx(full_bar, 3 * kBwBBytes);
      for (int q = 0; q < 3; ++q)
        for (int at = 0; at < kBwTN / 64; ++at)
          tma_load_2d(&maps.b, full_bar, b_base + q * kBwBBytes + at * (kBwK * 128), ab0 + 64 * at,
                      (q * npg + pg) * kBwK);
    }
    if (warp == 0) {
      tmem_alloc(smem_u32(tmem_slot), kBwTN);
      tmem_relinquish();
    }
    // the three parts of w: row r = pair p0 + r, 16-byte chunk c = kernel points 8c .. 8c + 7,
    // stored at r * 128 + ((c ^ r % 8) << 4) of each part (K-major, 128-byte swizzle)
#pragma unroll
    for (int e = 0; e < kBwTP * 8 / kBwThreads; ++e) {
      const int i = tid + kBwThreads * e, r = i >> 3, c = i & 7, p = p0 + r;
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = 0.f;
      if (p < npairs) {
        const int co = p / d.c_in, ci = p - co * d.c_in;
        const float* wr = w + ((((int64_t)co * d.s_out + s) * d.c_in + ci) * d.s_in + sp) * d.K;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (8 * c + j < d.K) x[j] = __ldg(wr + 8 * c + j);
      }
      uint32_t q0[4], q1[4], q2[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float lo = x[2 * j], hi = x[2 * j + 1];
        const __nv_bfloat16 l0 = __float2bfloat16_rn(lo), h0 = __float2bfloat16_rn(hi);
        lo -= __bfloat162float(l0);
        hi -= __bfloat162float(h0);
        const __nv_bfloat16 l1 = __float2bfloat16_rn(lo), h1 = __float2bfloat16_rn(hi);
        lo -= __bfloat162float(l1);
        hi -= __bfloat162float(h1);
        q0[j] = bf16_bits2(l0, h0);
        q1[j] = bf16_bits2(l1, h1);
        q2[j] = bf16_bits2(__float2bfloat16_rn(lo), __float2bfloat16_rn(hi));
      }
      const uint32_t off = (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
      *reinterpret_cast<uint4*>(smem + off) = make_uint4(q0[0], q0[1], q0[2], q0[3]);
      *reinterpret_cast<uint4*>(smem + kBwABytes + off) = make_uint4(q1[0], q1[1], q1[2], q1[3]);
      *reinterpret_cast<uint4*>(smem + 2 * kBwABytes + off) = make_uint4(q2[0], q2[1], q2[2], q2[3]);
    }
    fence_proxy_async_smem();  // the w parts, written by the threads, before the MMAs read them
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (tid == 0) {
      if (wait_bounded(full_bar, 0, abort_flag, err, kErrBwLoad)) {
        tc_fence_after();
        // A K-major (rows of 64 k, 8-row groups 1024 B apart, 16 k = 32 B per MMA); B MN-major
        // (64-entry atoms 8 KiB apart, 8-k groups 1024 B apart, 16 k = 2048 B per MMA)
        constexpr uint32_t idesc = idesc_bf16(kBwTP, kBwTN, false, true);
        bool first = true;
        for (int ti = 0; ti < 6; ++ti) {
          const int t = 5 - ti;  // smallest part products first
          const uint32_t asrc = a_base + bw_part_a(t) * kBwABytes, bsrc = b_base + bw_part_b(t) * kBwBBytes;
#pragma unroll
          for (int k = 0; k < kBwK / 16; ++k) {
            const uint64_t ad = umma_desc(asrc + k * 32, 16, 1024, kSwizzle128B);
            const uint64_t bd = umma_desc(bsrc + k * 2048, kBwK * 128, 1024, kSwizzle128B);
            mma_bf16(tmem_base, ad, bd, idesc, !first);
            first = false;
          }
        }
        mma_commit(done_bar);
      }
    }
    __syncwarp();
    ok = wait_bounded(done_bar, 0, abort_flag, err, kErrBwMma);
    tc_fence_after();
    // accumulator -> BF16 -> staging in W's order: warp w reads TMEM lanes 32 (w % 4) ..
    // (pairs) and kCols columns from kCols (w / 4) in 16-column loads
    if (__all_sync(0xffffffffu, ok)) {
      constexpr int kCols = kBwTN / (kBwThreads / 128);  // columns per warp
      const int quarter = warp & 3, cq = warp >> 2, prow = 32 * quarter + lane;
      const bool pv = prow < np;
      const int co_l = prow / d.c_in, ci = prow - co_l * d.c_in;
      const uint32_t tl = tmem_base + ((uint32_t)(32 * quarter) << 16);
      __nv_bfloat16* srow = stg + ((int64_t)co_l * na * d.c_in + ci) * d.n_in;  // + (a - a_lo) rowlen + b
#pragma unroll 1
      for (int c = 0; c < kCols; c += 16) {
        const int col = kCols * cq + c;
        uint32_t r[16];
        tmem_ld16_nowait(tl + (uint32_t)col, r);
        tmem_wait_ld();
        const int ab = ab0 + col;
        int a = ab / d.n_in, b = ab - a * d.n_in;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          if (pv && col + jj < nabc) srow[(a - a_lo) * rowlen + b] = __float2bfloat16_rn(__uint_as_float(r[jj]));
          if (++b == d.n_in) {
            b = 0;
            ++a;
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      tmem_dealloc(tmem_base, kBwTN);
    }
  }
  // copy-out: run (co, a) of W's row (s, co, a), columns s' in_blk + (ci, b), from staging
  // row (co - co_lo, a - a_lo); whole runs in 16-byte chunks when vec, partial ones (the
  // tile's first and last a) entry by entry
  const bool have = in_win && ok;
  for (int r = warp; r < nco * na; r += kBwThreads / 32) {
    const int co_l = r / na, a_l = r - co_l * na, co = co_lo + co_l, aa = a_lo + a_l;
    const int b0 = max(0, ab0 - aa * d.n_in), b1 = min(d.n_in, ab0 + nabc - aa * d.n_in);
    __nv_bfloat16* dst = W + (((int64_t)s * d.c_out + co) * d.n_out + aa) * d.ldW + (int64_t)sp * d.in_blk;
    const __nv_bfloat16* src = stg + (int64_t)r * rowlen;
    if (b0 == 0 && b1 == d.n_in) {
      if (vec) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int j = lane; j < rowlen / 8; j += 32)
          reinterpret_cast<uint4*>(dst)[j] = have ? reinterpret_cast<const uint4*>(src)[j] : z;
      } else {
        for (int j = lane; j < rowlen; j += 32) dst[j] = have ? src[j] : __float2bfloat16_rn(0.f);
      }
    } else {
      int bj = lane % d.n_in;
      for (int j = lane; j < rowlen; j += 32) {
        if (bj >= b0 && bj < b1) dst[j] = have ? src[j] : __float2bfloat16_rn(0.f);
        bj += 32;
        while (bj >= d.n_in) bj -= d.n_in;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 bw_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

constexpr size_t kBwSmem = 1024 + kBwOpBytes + 64;

}  // namespace

cudaError_t build_w_tables_create(const LscDims& dt, const float* d_M, BuildWTables& t, std::string& err) {
  t = BuildWTables();
  const int npg = dt.s_out * dt.s_in, nab = dt.n_out * dt.n_in;
  // the staging tile: up to 128 pairs x bw_max_rows(n_in) rows of n_in entries, in the operand space
  if (dt.K > kBwK || npg < 1 || nab < 1 || (size_t)kBwTP * bw_max_rows(dt.n_in) * dt.n_in * 2 > kBwOpBytes)
    return cudaSuccess;  // the CUDA-core build takes these
  t.npg = npg;
  t.ldm = (nab + 63) / 64 * 64;
  const size_t part = (size_t)npg * kBwK * t.ldm;
  void* mp = nullptr;
  cudaError_t e = cudaMalloc(&mp, 3 * part * 2);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)std::min<size_t>((part + 255) / 256, 152 * 8);
    split_m_kernel<<<blocks, 256>>>(dt, d_M, static_cast<__nv_bfloat16*>(mp), t.ldm, npg);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    if (mp) cudaFree(mp);
    t = BuildWTables();
    return e;
  }
  t.d_mp = mp;
  t.ok = true;
  return cudaSuccess;
}

void build_w_tables_destroy(BuildWTables& t) {
  if (t.d_mp) cudaFree(t.d_mp);
  t = BuildWTables();
}

bool tc_build_w_supported(const LscDims& d, const BuildWTables& t) {
  if (!tc_enabled() || !t.ok || d.K > kBwK || !bw_encode()) return false;
  if (d.s_out * d.s_in != t.npg || d.c_in < 1 || kBwTP % d.c_in != 0) return false;
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  return major == 10;
}

cudaError_t tc_build_w(const LscDims& d, const BuildWTables& t, const float* w, void* W, int* err, cudaStream_t st) {
  TraceScope trace("lsc_build_w_tc", st);
  const int npg = d.s_out * d.s_in, nab = d.n_out * d.n_in;
  cudaError_t e;
  // padding columns between shell blocks stay zero
  if (d.in_blk != (int64_t)d.c_in * d.n_in) {
    e = cudaMemsetAsync(W, 0, (size_t)d.rows_out * d.ldW * 2, st);
    if (e != cudaSuccess) return e;
  }
  BwMaps maps;
  memset(&maps, 0, sizeof maps);
  {
    const cuuint64_t dims[2] = {(cuuint64_t)t.ldm, (cuuint64_t)(3 * npg * kBwK)};
    const cuuint64_t strides[1] = {(cuuint64_t)t.ldm * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kBwK};
    const cuuint32_t es[2] = {1, 1};
    if (bw_encode()(&maps.b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t.d_mp, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  // whole runs in 16-byte chunks: W 16-byte aligned, rows and shell blocks of multiples of 8
  const int rowlen = d.c_in * d.n_in;
  const int vec = (reinterpret_cast<uintptr_t>(W) & 15u) == 0 && rowlen % 8 == 0 && d.ldW % 8 == 0 && d.in_blk % 8 == 0;
  e = cudaFuncSetAttribute(build_w_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwSmem);
  if (e != cudaSuccess) return e;
  const int npairs = d.c_out * d.c_in;
  const dim3 grid((unsigned)((nab + kBwTN - 1) / kBwTN), (unsigned)((npairs + kBwTP - 1) / kBwTP), (unsigned)npg);
  build_w_tc_kernel<<<grid, kBwThreads, kBwSmem, st>>>(maps, d, w, static_cast<__nv_bfloat16*>(W), vec, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace delimit
