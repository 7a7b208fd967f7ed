// tcgen05 grouped transforms with FP32 activations: Signal2SH, SH2Signal and their
// adjoints (Sec. 2.2) at FP32 accuracy on the BF16 tensor cores.  Per shell g and
// channel c:
//   Y[(g,c,i), v] = sum_j T_g[i][j] X[(g,c,j), v]
// Every FP32 value is the sum of three BF16 parts (x = x0 + x1 + x2, each part the
// BF16 rounding of what the earlier ones leave, to 2^-27 |x|); so is every operator
// entry (T = T0 + T1 + T2, split once on the host).  The six part products xi Tj
// with i + j <= 2 (the three dropped ones are below 2^-26 of the leading one) are
// accumulated in FP32 in TMEM, smallest first.
//
// Data path per 128-voxel tile, in chunks of 32 input rows: TMA copies each FP32
// chunk (32 rows x 128 voxels, as four 128-byte-swizzled boxes of 32 voxels) into a ring
// of raw stages in shared memory; four converter warps split every value into its three BF16 parts and write them in the
// 128-byte-swizzled MN-major layout the MMA reads; one thread issues the MMAs; four
// epilogue warps read the accumulator from TMEM and store the outputs (voxels
// contiguous, 128-byte rows per warp).  Only the input is read from and only the
// output is written to HBM.  Each CTA serves one shell group (the SMs split across
// groups in proportion to their bytes), so only that group's three operator images are
// resident; tiles, chunks and stages advance in 32-bit steps (no divisions in the loops).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace delimit {

namespace {

constexpr int kConvWarps = 4;
constexpr int kEpiWarps = 4;  // one per TMEM lane quarter
constexpr int kThreads = 32 * (2 + kConvWarps + kEpiWarps);
constexpr int kMaxG = 8;
constexpr int kAccCols = 256;                           // TMEM columns per accumulator buffer
constexpr int kChunkRows = 32;                          // input rows per chunk
constexpr int kRowsPerWarp = kChunkRows / kConvWarps;   // rows each converter warp splits per chunk
constexpr uint32_t kRawBytes = kChunkRows * 128 * 4;    // 16 KiB FP32 chunk
constexpr uint32_t kPlaneBytes = kChunkRows * 128 * 2;  // 8 KiB per BF16 part
constexpr uint32_t kStageBytes = 3 * kPlaneBytes;       // 24 KiB
constexpr size_t kSmemLimit = 227 * 1024;

enum : int {
  kErrRawFull = 0x3100,
  kErrRawEmpty = 0x3200,
  kErrPlFull = 0x3300,
  kErrPlEmpty = 0x3400,
  kErrTFull = 0x3500,
  kErrTEmpty = 0x3600,
  kErrDrain = 0x3700
};

}  // namespace

struct Tf32Group {
  int64_t x_row0, x_cstride, y_row0, y_cstride;
  int n_in, n_out, n_mma, kpad, npad, nchunks;
  int pstride;     // column offset between the operator parts (a multiple of 64)
  int cta0, ncta;  // the CTAs [cta0, cta0 + ncta) serve this group
};

struct Tf32Params {
  CUtensorMap mapA[kMaxG];  // FP32 input, 3-D {voxels, n_in rows, channels}, box {32, 32, 1}, 128-byte swizzle
  CUtensorMap mapB[kMaxG];  // operator parts side by side [kpad rows][npad], box {64, kpad}, 128-byte swizzle
  Tf32Group g[kMaxG];
  int n_groups, channels, m_tiles, raw_stages, pl_stages;
  uint32_t b_region;  // bytes reserved for one group's three images (1 KiB multiple)
  int64_t n_vox, ldx, ldy;
  const float* X;
  void* Y;
  int* err;
};

// part products (a, b) of x_a T_b, smallest first
__constant__ int8_t kProdA[6] = {2, 1, 0, 1, 0, 0};
__constant__ int8_t kProdB[6] = {0, 1, 2, 0, 1, 0};

// (x, y) -> BF16 parts packed in pairs: x = x0 + x1 + x2 and y likewise, each part the
// round-to-nearest BF16 of what the earlier ones leave (the differences are exact in FP32);
// p[q] holds part q of x in its low and of y in its high half
__device__ __forceinline__ void split3x2(float x, float y, uint32_t (&p)[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    p[q] = *reinterpret_cast<const uint32_t*>(&h);
    if (q < 2) {
      x -= __uint_as_float(p[q] << 16);
      y -= __uint_as_float(p[q] & 0xFFFF0000u);
    }
  }
}

// (tile, chunk) of a CTA's work in 32-bit steps: tile t = local + k * ncta = c * m_tiles + mt
struct Walk {
  int k, ch, c, mt;
  int nch, m_tiles, dc, dmt;
  // tiles t0, t0 + step, t0 + 2 step, ...
  __device__ __forceinline__ void init(int t0, int step, int nch_, int m_tiles_) {
    nch = nch_;
    m_tiles = m_tiles_;
    dc = step / m_tiles;
    dmt = step - dc * m_tiles;
    k = 0;
    ch = 0;
    c = t0 / m_tiles;
    mt = t0 - c * m_tiles;
  }
  __device__ __forceinline__ void next_chunk() {
    if (++ch < nch) return;
    ch = 0;
    next_tile();
  }
  __device__ __forceinline__ void next_tile() {
    ++k;
    c += dc;
    mt += dmt;
    if (mt >= m_tiles) {
      mt -= m_tiles;
      ++c;
    }
  }
};

// stage ring position: index and phase parity
struct Ring {
  int i, n;
  uint32_t ph;
  __device__ __forceinline__ void init(int n_) {
    i = 0;
    n = n_;
    ph = 0;
  }
  __device__ __forceinline__ void next() {
    if (++i == n) {
      i = 0;
      ph ^= 1u;
    }
  }
};

template <bool OUT_F32>
__global__ void __launch_bounds__(kThreads, 1) transform_tc_f32_kernel(const __grid_constant__ Tf32Params p) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int R = p.raw_stages, S = p.pl_stages;
  // layout: [B images (b_region)][raw FP32 chunks R x 16 KiB][part planes S x 24 KiB][barriers]
  const uint32_t sbase = smem_u32(smem);
  const uint32_t raw_base = sbase + p.b_region;
  const uint32_t pl_base = raw_base + (uint32_t)R * kRawBytes;
  const uint8_t* raw_ptr = smem + p.b_region;
  uint8_t* pl_ptr = smem + p.b_region + (size_t)R * kRawBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(pl_ptr + (size_t)S * kStageBytes);
  // bars: raw_full[R], raw_empty[R], pl_full[S], pl_empty[S], tfull[2], tempty[2], bload, drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * R + 2 * S + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  auto raw_full = [&](int r) { return smem_u32(bars + r); };
  auto raw_empty = [&](int r) { return smem_u32(bars + R + r); };
  auto pl_full = [&](int s) { return smem_u32(bars + 2 * R + s); };
  auto pl_empty = [&](int s) { return smem_u32(bars + 2 * R + S + s); };
  auto tfull = [&](int b) { return smem_u32(bars + 2 * R + 2 * S + b); };
  auto tempty = [&](int b) { return smem_u32(bars + 2 * R + 2 * S + 2 + b); };
  const uint32_t bload_bar = smem_u32(bars + 2 * R + 2 * S + 4);
  const uint32_t drain_bar = smem_u32(bars + 2 * R + 2 * S + 5);

  // this CTA's group and its tiles t = local, local + ncta, ... < channels * m_tiles
  int gi = p.n_groups - 1;
  while (gi > 0 && (int)blockIdx.x < p.g[gi].cta0) --gi;
  const Tf32Group& G = p.g[gi];
  const int local = (int)blockIdx.x - G.cta0;
  const int n_tiles = p.channels * p.m_tiles;  // < 2^31 / nchunks (checked on the host)
  const int my_tiles = local < G.ncta ? (n_tiles - local + G.ncta - 1) / G.ncta : 0;
  const int nch = G.nchunks;

  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r) {
      mbar_init(raw_full(r), 1);
      mbar_init(raw_empty(r), kConvWarps);
    }
    for (int s = 0; s < S; ++s) {
      mbar_init(pl_full(s), kConvWarps);
      mbar_init(pl_empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), kEpiWarps);
    }
    mbar_init(bload_bar, 1);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), 2 * kAccCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0 && my_tiles > 0) {
      // the group's operator parts, then the raw FP32 input chunks
      mbar_arrive_expect_tx(bload_bar, (uint32_t)(G.kpad * G.npad * 2));
      for (int j = 0; j < G.npad / 64; ++j)
        tma_load_2d(&p.mapB[gi], bload_bar, sbase + j * G.kpad * 128, j * 64, 0);
      int pend[8];
      for (int r = 0; r < 8; ++r) pend[r] = -1;
      Walk w;
      w.init(local, G.ncta, nch, p.m_tiles);
      Ring rr;
      rr.init(R);
      for (; w.k < my_tiles; w.next_chunk()) {
        if (!wait_bounded(raw_empty(rr.i), rr.ph ^ 1u, abort_flag, p.err, kErrRawEmpty)) break;
        mbar_arrive_expect_tx(raw_full(rr.i), kRawBytes);
        // four boxes of 32 voxels x 32 rows, 128-byte swizzled: box b at b * 4 KiB
#pragma unroll
        for (int b = 0; b < 4; ++b)
          tma_load_3d(&p.mapA[gi], raw_full(rr.i), raw_base + rr.i * kRawBytes + b * (kRawBytes / 4), w.mt * 128 + 32 * b,
                      w.ch * kChunkRows, w.c);
        pend[rr.i] = (int)rr.ph;
        rr.next();
      }
      wait_drain(bload_bar, 0, p.err, kErrDrain);
      for (int r = 0; r < R; ++r)
        if (pend[r] >= 0) wait_drain(raw_full(r), (uint32_t)pend[r], p.err, kErrDrain);
    }
  } else if (warp == 1) {
    if (lane == 0 && my_tiles > 0) {
      const int ksteps = G.kpad / 16;
      const uint32_t idesc = idesc_bf16(128, G.n_mma, true, true);
      // operator part q starts at column q * pstride: 64-column atoms are kpad * 128 bytes apart
      const uint32_t part_bytes = (uint32_t)(G.pstride / 64 * G.kpad * 128);
      bool ok = wait_bounded(bload_bar, 0, abort_flag, p.err, kErrPlFull);
      Ring ss;
      ss.init(S);
      for (int k = 0; ok && k < my_tiles; ++k) {
        const int acc = k & 1;
        if (!wait_bounded(tempty(acc), (uint32_t)((k >> 1) & 1) ^ 1u, abort_flag, p.err, kErrTEmpty)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kAccCols);
        for (int ch = 0; ch < nch; ++ch) {
          if (!wait_bounded(pl_full(ss.i), ss.ph, abort_flag, p.err, kErrPlFull)) {
            ok = false;
            break;
          }
          tc_fence_after();
          constexpr int kKs = kChunkRows / 16;  // k-steps of 16 rows per chunk
          const int kk_n = min(kKs, ksteps - kKs * ch);
          for (int kk = 0; kk < kk_n; ++kk) {
            const int kg = kKs * ch + kk;  // k-step of 16 rows within the whole K
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
              const uint64_t ad = umma_desc(pl_base + ss.i * kStageBytes + kProdA[pr] * kPlaneBytes + kk * 2048,
                                            kChunkRows * 128, 1024, kSwizzle128B);
              const uint64_t bd = umma_desc(sbase + kProdB[pr] * part_bytes + kg * 2048, G.kpad * 128, 1024,
                                            kSwizzle128B);
              mma_bf16(d_tmem, ad, bd, idesc, (ch | kk | pr) != 0);
            }
          }
          mma_commit(pl_empty(ss.i));
          ss.next();
        }
        if (!ok) break;
        mma_commit(tfull(acc));
      }
      mma_commit(drain_bar);
      wait_drain(drain_bar, 0, p.err, kErrDrain);
    }
  } else if (warp < 2 + kConvWarps) {
    // converters: warp cw splits rows cw * kRowsPerWarp ... of every raw chunk; lane l holds voxels
    // 4l .. 4l + 3 (a 16-byte read from the swizzled boxes, conflict-free) and writes 8 bytes of each
    // part plane: voxel half l / 16, 16-byte chunk (l % 16) / 2 XOR row % 8, half-chunk l % 2
    const int cw = warp - 2;
    const int half = lane >> 4, sub = lane & 1, c16 = (lane & 15) >> 1;
    Ring rr, ss;
    rr.init(R);
    ss.init(S);
    const int n_chunks = my_tiles * nch;
    for (int i = 0; i < n_chunks; ++i) {
      bool w_ok = wait_bounded_sleep(raw_full(rr.i), rr.ph, abort_flag, p.err, kErrRawFull);
      w_ok = w_ok && wait_bounded_sleep(pl_empty(ss.i), ss.ph ^ 1u, abort_flag, p.err, kErrPlEmpty);
      if (!__all_sync(0xffffffffu, w_ok)) break;
      const float* src = reinterpret_cast<const float*>(raw_ptr + (size_t)rr.i * kRawBytes);
      uint8_t* dst = pl_ptr + (size_t)ss.i * kStageBytes;
#pragma unroll
      for (int k2 = 0; k2 < kRowsPerWarp; ++k2) {
        const int row = cw * kRowsPerWarp + k2;  // row within the chunk
        // voxels 4l .. 4l + 3: box l / 8, 16-byte chunk (l % 8) XOR row % 8 of its 128-byte row
        const float4 v = *reinterpret_cast<const float4*>(src + (lane >> 3) * (kChunkRows * 32) + row * 32 +
                                                          (((lane & 7) ^ (row & 7)) << 2));
        uint32_t lo[3], hi[3];
        split3x2(v.x, v.y, lo);
        split3x2(v.z, v.w, hi);
        const uint32_t off = (uint32_t)(half * kChunkRows * 128 + row * 128 + ((c16 ^ (row & 7)) << 4) + sub * 8);
#pragma unroll
        for (int q = 0; q < 3; ++q) *reinterpret_cast<uint2*>(dst + q * kPlaneBytes + off) = make_uint2(lo[q], hi[q]);
      }
      // the planes are read by the tensor cores (async proxy); the raw chunk is free again
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(pl_full(ss.i));
        mbar_arrive(raw_empty(rr.i));
      }
      rr.next();
      ss.next();
    }
  } else {
    // epilogue: TMEM lane quarter q holds voxels 32q .. 32q + 31 of the tile; each thread
    // stores its voxel's outputs (a warp writes 128 contiguous bytes per output row)
    const int q = warp & 3;
    Walk w;
    w.init(local, G.ncta, 1, p.m_tiles);
    for (; w.k < my_tiles; w.next_tile()) {
      const int k = w.k, c = w.c, mt = w.mt;
      const int acc = k & 1;
      const bool ok = wait_bounded_sleep(tfull(acc), (uint32_t)((k >> 1) & 1), abort_flag, p.err, kErrTFull);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int64_t v = (int64_t)mt * 128 + q * 32 + lane;
      const bool in = v < p.n_vox;
      const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kAccCols);
      // this voxel's element of output row (y_row0 + c * y_cstride + col), column by column
      const int64_t e0 = (G.y_row0 + (int64_t)c * G.y_cstride) * p.ldy + v;
      for (int c0 = 0; c0 < G.n_mma; c0 += 32) {
        uint32_t rv[2][16];
        tmem_ld16_nowait(tl + (uint32_t)c0, rv[0]);
        if (c0 + 16 < G.n_mma) tmem_ld16_nowait(tl + (uint32_t)(c0 + 16), rv[1]);
        tmem_wait_ld();
        if (in) {
          if (OUT_F32) {
            float* y = reinterpret_cast<float*>(p.Y) + e0 + (int64_t)c0 * p.ldy;
#pragma unroll
            for (int j = 0; j < 32; ++j, y += p.ldy)
              if (c0 + j < G.n_out) __stcs(y, __uint_as_float(rv[j >> 4][j & 15]));
          } else {
            __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(p.Y) + e0 + (int64_t)c0 * p.ldy;
#pragma unroll
            for (int j = 0; j < 32; ++j, y += p.ldy)
              if (c0 + j < G.n_out) *y = __float2bfloat16_rn(__uint_as_float(rv[j >> 4][j & 15]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(acc));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * kAccCols);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 f32_encode() {
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

struct DevProps {
  int sms = 0, major = 0;
};

DevProps f32_dev() {
  DevProps d;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev);
  d.sms = std::max(1, d.sms);
  return d;
}

int rup(int x, int a) { return (x + a - 1) / a * a; }

// shared memory of a launch with R raw and S plane stages and a B region of `b_region` bytes
size_t f32_smem(uint32_t b_region, int R, int S) {
  return 1024 + (size_t)b_region + (size_t)R * kRawBytes + (size_t)S * kStageBytes + (2 * R + 2 * S + 6) * 8 + 16;
}

uint32_t b_region_bytes(const TcBasisTables& t, int kind) {
  uint32_t mx = 0;
  for (int s = 0; s < t.n_shells; ++s) mx = std::max(mx, (uint32_t)(t.kpad[s][kind] * t.npad3[s][kind] * 2));
  return (mx + 1023) / 1024 * 1024;
}

}  // namespace

cudaError_t tc_basis_tables_create_f32(const BasisHost& h, TcBasisTables& t, std::string& err) {
  t.ok3 = false;
  t.d_mem3 = nullptr;
  if (!t.ok) return cudaSuccess;  // no tensor-core images at all (too many shells)
  // three BF16 parts of every operator T (T = T0 + T1 + T2, each the rounding of what is
  // left), side by side along the output axis (row k = input index, column = part offset +
  // output index) so that one MMA can multiply an activation part by several operator parts
  std::vector<__nv_bfloat16> img;
  for (int s = 0; s < t.n_shells; ++s) {
    const ShellHost& sh = h.shells[s];
    for (int kind = 0; kind < 4; ++kind) {
      const int n_in = t.n_in[s][kind], n_out = t.n_out[s][kind], kpad = t.kpad[s][kind];
      const int n1 = rup(n_out, 16);
      const int pstride = rup(n1, 64);  // column offset of part q: q * pstride (whole 64-column atoms)
      const int npad = 3 * pstride;
      t.npad3[s][kind] = npad;
      auto T = [&](int i, int j) -> double {
        switch (kind) {
          case 0: return sh.P[size_t(i) * sh.m + j];   // P [N][m]
          case 1: return sh.B[size_t(i) * h.N + j];    // B [m][N]
          case 2: return sh.P[size_t(j) * sh.m + i];   // P^T [m][N]
          default: return sh.B[size_t(j) * h.N + i];   // B^T [N][m]
        }
      };
      const size_t off = (img.size() + 511) / 512 * 512;  // 1 KiB aligned
      img.resize(off + size_t(kpad) * npad, __float2bfloat16_rn(0.f));
      for (int k = 0; k < n_in; ++k)
        for (int n = 0; n < n_out; ++n) {
          double rest = T(n, k);
          for (int q = 0; q < 3; ++q) {
            const __nv_bfloat16 part = __float2bfloat16_rn(float(rest));
            img[off + size_t(k) * npad + q * pstride + n] = part;
            rest -= double(__bfloat162float(part));
          }
        }
      t.off3[s][kind] = off * 2;
    }
  }
  cudaError_t e = cudaMalloc(&t.d_mem3, img.size() * 2);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    t.d_mem3 = nullptr;
    return e;
  }
  e = cudaMemcpy(t.d_mem3, img.data(), img.size() * 2, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    cudaFree(t.d_mem3);
    t.d_mem3 = nullptr;
    return e;
  }
  t.ok3 = true;
  return cudaSuccess;
}

void tc_basis_tables_destroy_f32(TcBasisTables& t) {
  if (t.d_mem3) cudaFree(t.d_mem3);
  t.d_mem3 = nullptr;
  t.ok3 = false;
}

bool tc_transform_f32_supported(const TcBasisTables& t, int kind, int out_t) {
  if (!t.ok3 || !tc_enabled() || !f32_encode() || t.n_shells > kMaxG) return false;
  if (f32_dev().major != 10) return false;
  for (int s = 0; s < t.n_shells; ++s)
    if (t.n_in[s][kind] > 256 || t.n_out[s][kind] > 256) return false;
  (void)out_t;
  return f32_smem(b_region_bytes(t, kind), 2, 2) <= kSmemLimit;
}

cudaError_t tc_transform_f32_launch(const TcBasisTables& t, int kind, const float* X, void* Y, int64_t n_vox, int C,
                                    int64_t ldx, int64_t ldy, int out_t, int* err_word, cudaStream_t st) {
  auto fn = f32_encode();
  if (!fn) return cudaErrorNotSupported;
  static const char* kNames[4] = {"signal2sh_tc_f32", "sh2signal_tc_f32", "signal2sh_bwd_tc_f32",
                                  "sh2signal_bwd_tc_f32"};
  TraceScope trace(kNames[kind & 3], st);
  Tf32Params p;
  memset(&p, 0, sizeof p);
  const bool x_is_sig = (kind == 0 || kind == 3);  // input rows in the signal layout
  const int m_tiles = (int)((n_vox + 127) / 128);
  const int64_t n_tiles = (int64_t)C * m_tiles;
  // the kernel walks tiles and chunks in 32 bits
  if (n_tiles * ((int64_t)256 / kChunkRows + 1) >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  double work[kMaxG], tot = 0;
  for (int s = 0; s < t.n_shells; ++s) {
    const int n_in = t.n_in[s][kind], n_out = t.n_out[s][kind], kpad = t.kpad[s][kind];
    const int64_t sig_row0 = int64_t(C) * t.dir_off[s], sig_cs = t.m[s];
    const int64_t sh_row0 = int64_t(s) * C * t.N, sh_cs = t.N;
    const int64_t x_row0 = x_is_sig ? sig_row0 : sh_row0, x_cs = x_is_sig ? sig_cs : sh_cs;
    Tf32Group& G = p.g[s];
    G.x_row0 = x_row0;
    G.x_cstride = x_cs;
    G.n_in = n_in;
    G.y_row0 = x_is_sig ? sh_row0 : sig_row0;
    G.y_cstride = x_is_sig ? sh_cs : sig_cs;
    G.n_out = n_out;
    G.n_mma = rup(n_out, 16);
    G.kpad = kpad;
    G.npad = t.npad3[s][kind];
    G.pstride = rup(G.n_mma, 64);
    G.nchunks = (kpad + kChunkRows - 1) / kChunkRows;
    work[s] = double(n_in + n_out);  // bytes per voxel-channel, the HBM-bound cost
    tot += work[s];
    {  // A: FP32 input, 3-D {voxels, rows of one channel, channels}; rows past n_in read as zero
      const char* base = reinterpret_cast<const char*>(X) + x_row0 * ldx * 4;
      cuuint64_t dims[3] = {(cuuint64_t)n_vox, (cuuint64_t)n_in, (cuuint64_t)C};
      cuuint64_t strides[2] = {(cuuint64_t)ldx * 4, (cuuint64_t)(x_cs * ldx * 4)};
      cuuint32_t box[3] = {32, (cuuint32_t)kChunkRows, 1};
      cuuint32_t es[3] = {1, 1, 1};
      if (fn(&p.mapA[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<char*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
    {  // B: the operator parts side by side, [kpad][npad3]
      const int npad3 = t.npad3[s][kind];
      const char* base = static_cast<const char*>(t.d_mem3) + t.off3[s][kind];
      cuuint64_t dims[2] = {(cuuint64_t)npad3, (cuuint64_t)kpad};
      cuuint64_t strides[1] = {(cuuint64_t)npad3 * 2};
      cuuint32_t box[2] = {64, (cuuint32_t)kpad};
      cuuint32_t es[2] = {1, 1};
      if (fn(&p.mapB[s], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<char*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
  }
  // one CTA per SM, the SMs split across the groups in proportion to their bytes
  // (largest remainders; every group at least one CTA, none more than its tile count)
  const DevProps dp = f32_dev();
  const int G_n = t.n_shells;
  const int total = (int)std::max<int64_t>(G_n, std::min<int64_t>(dp.sms, n_tiles * G_n));
  int ncta[kMaxG];
  double frac[kMaxG];
  int used = 0;
  for (int s = 0; s < G_n; ++s) {
    const double share = total * work[s] / tot;
    ncta[s] = std::max(1, (int)std::floor(share));
    frac[s] = share - std::floor(share);
    used += ncta[s];
  }
  while (used > total) {  // groups raised to one CTA: take the surplus from the largest
    int big = 0;
    for (int s = 1; s < G_n; ++s)
      if (ncta[s] > ncta[big]) big = s;
    --ncta[big];
    --used;
  }
  while (used < total) {  // hand out the rest by largest remainder
    int best = 0;
    for (int s = 1; s < G_n; ++s)
      if (frac[s] > frac[best]) best = s;
    ++ncta[best];
    frac[best] = -1.0;
    ++used;
  }
  int cta0 = 0;
  for (int s = 0; s < G_n; ++s) {
    p.g[s].cta0 = cta0;
    p.g[s].ncta = (int)std::min<int64_t>(ncta[s], n_tiles);
    cta0 += p.g[s].ncta;
  }
  p.n_groups = t.n_shells;
  p.channels = C;
  p.m_tiles = m_tiles;
  p.b_region = b_region_bytes(t, kind);
  // two part-plane stages (the MMAs drain them quickly), then as many raw chunks as fit,
  // up to 8: the bytes in flight from HBM are what the kernel's speed depends on
  int R = 8, S = 2;
  while (R > 2 && f32_smem(p.b_region, R, S) > kSmemLimit) --R;
  if (f32_smem(p.b_region, R, S) > kSmemLimit) return cudaErrorInvalidValue;
  p.raw_stages = R;
  p.pl_stages = S;
  p.n_vox = n_vox;
  p.ldx = ldx;
  p.ldy = ldy;
  p.X = X;  // (read through mapA)
  p.Y = Y;
  p.err = err_word;
  // at least 120 KiB so that two CTAs never share an SM (each holds 512 TMEM columns)
  const size_t smem = std::max<size_t>(120 * 1024, f32_smem(p.b_region, R, S));
  auto kern = out_t == 0 ? transform_tc_f32_kernel<true> : transform_tc_f32_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<cta0, kThreads, smem, st>>>(p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace delimit
