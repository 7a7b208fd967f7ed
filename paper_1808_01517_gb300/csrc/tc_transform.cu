// tcgen05 + TMA grouped transforms of the BF16 path: Signal2SH, SH2Signal and
// their adjoints (Sec. 2.2).  Per shell g and channel c:
//   Y[(g,c,i), v] = sum_j T_g[i][j] X[(g,c,j), v]
// D[voxel, i] lives in TMEM (M = 128 voxels, N = n_out rounded to 16); A is a
// 128-voxel x n_in tile of X loaded by TMA through a 3-D map {voxels, rows,
// channels} so rows past n_in are zero-filled per channel; B = T_g^T (BF16,
// [n_in padded to 16] x [n_out padded to 64]) stays resident in shared memory.
// The kernel is HBM-bound (about 15 FLOP per byte at order 8): each CTA keeps
// STAGES A tiles in flight and double-buffers the accumulator.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace delimit {

namespace {

constexpr int kEpiWarps = 8;                 // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // + TMA warp + MMA warp
constexpr int kMaxTcGroups = 8;
constexpr int kAccCols = 256;  // TMEM columns per accumulator buffer

enum : int { kErrFull = 0x1100, kErrEmpty = 0x1200, kErrTFull = 0x1300, kErrTEmpty = 0x1400, kErrDrain = 0x1500 };

}  // namespace

struct TfGroup {
  int64_t y_row0, y_cstride;
  int n_out, n_mma, kpad, npad;
  uint32_t b_off;  // byte offset of this group's B image in shared memory
};

struct TfParams {
  CUtensorMap mapA[kMaxTcGroups];
  CUtensorMap mapB[kMaxTcGroups];
  CUtensorMap mapY[kMaxTcGroups];  // output, 3-D {voxels, rows of one channel, channels}
  TfGroup g[kMaxTcGroups];
  int n_groups, channels, m_tiles, stages, stage_bytes, stg_bytes;
  int swz;  // launch the SWZ instantiation (wide BF16 outputs)
  uint32_t b_total;
  int64_t total_tiles, n_vox, ldy;
  void* Y;
  int* err;
};

// Tile t = (g * C + c) * M + mt walked with a stride of gridDim.x: the stride is
// split into (dg, dc, dmt) once, so each step costs a few adds and compares
// instead of the 64-bit divisions a fresh decode takes (per tile, on the single
// threads that issue the copies and the MMAs).
struct TileIter {
  uint32_t g, c, mt, dg, dc, dmt, C, M;
  __device__ __forceinline__ void init(uint32_t t0, uint32_t step, uint32_t C_, uint32_t M_) {
    C = C_;
    M = M_;
    const uint32_t pg = C * M;
    g = t0 / pg;
    uint32_t r = t0 - g * pg;
    c = r / M;
    mt = r - c * M;
    dg = step / pg;
    r = step - dg * pg;
    dc = r / M;
    dmt = r - dc * M;
  }
  __device__ __forceinline__ void next() {
    mt += dmt;
    c += dc;
    g += dg;
    if (mt >= M) {
      mt -= M;
      ++c;
    }
    if (c >= C) {
      c -= C;
      ++g;
    }
  }
};

// SWZ: BF16 output through stmatrix into 128-byte-swizzled staging halves (a separate
// instantiation, so that the one-box epilogue keeps its own register allocation)
template <bool OUT_F32, bool SWZ>
__global__ void __launch_bounds__(kThreads, 1) transform_tc_kernel(const __grid_constant__ TfParams p) {
  static_assert(!(OUT_F32 && SWZ), "the swizzled epilogue writes BF16");
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int STAGES = p.stages;
  // layout: [B images][A stages][2 output staging tiles [n_mma rows][128 voxels]][barriers]
  const uint32_t sbase = smem_u32(smem);
  const uint32_t a_base = sbase + p.b_total;
  const uint32_t stg_base = a_base + STAGES * p.stage_bytes;
  uint8_t* stg_ptr = smem + p.b_total + (size_t)STAGES * p.stage_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_ptr + 2 * (size_t)p.stg_bytes);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], bload, drain, stg_ready[2], stg_free[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 10);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto tfull_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };
  const uint32_t bload_bar = smem_u32(bars + 2 * STAGES + 4);
  const uint32_t drain_bar = smem_u32(bars + 2 * STAGES + 5);
  auto stg_ready_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 6 + b); };
  auto stg_free_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 8 + b); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kEpiWarps);
    }
    mbar_init(bload_bar, 1);
    mbar_init(drain_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(stg_ready_bar(b), kEpiWarps);
      mbar_init(stg_free_bar(b), 1);
    }
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
  const uint32_t total = (uint32_t)p.total_tiles;  // < 2^31 (checked on the host)

  if (warp == 0 && lane == 0) {
    // resident B images (all groups), then the A ring
    uint32_t bbytes = 0;
    for (int g = 0; g < p.n_groups; ++g) bbytes += (uint32_t)(p.g[g].kpad * p.g[g].npad * 2);
    mbar_arrive_expect_tx(bload_bar, bbytes);
    for (int g = 0; g < p.n_groups; ++g)
      for (int j = 0; j < p.g[g].npad / 64; ++j)
        tma_load_2d(&p.mapB[g], bload_bar, sbase + p.g[g].b_off + j * p.g[g].kpad * 128, j * 64, 0);
    int stage = 0;
    uint32_t phase = 0;
    int pend[8];
    for (int s = 0; s < 8; ++s) pend[s] = -1;
    TileIter ti;
    ti.init(blockIdx.x, gridDim.x, (uint32_t)p.channels, (uint32_t)p.m_tiles);
    for (uint32_t t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ti.next()) {
      const int g = (int)ti.g, c = (int)ti.c, mt = (int)ti.mt;
      if (!wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, p.err, kErrEmpty)) break;
      const uint32_t dst = a_base + stage * p.stage_bytes;
      const int kp = p.g[g].kpad;
      mbar_arrive_expect_tx(full_bar(stage), (uint32_t)(2 * kp * 128));
      tma_load_3d(&p.mapA[g], full_bar(stage), dst, mt * 128, 0, c);
      tma_load_3d(&p.mapA[g], full_bar(stage), dst + kp * 128, mt * 128 + 64, 0, c);
      pend[stage] = (int)phase;
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    wait_drain(bload_bar, 0, p.err, kErrDrain);
    for (int s = 0; s < STAGES; ++s)
      if (pend[s] >= 0) wait_drain(full_bar(s), (uint32_t)pend[s], p.err, kErrDrain);
  } else if (warp == 1 && lane == 0) {
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool bready = wait_bounded(bload_bar, 0, abort_flag, p.err, kErrFull);
    TileIter ti;
    ti.init(blockIdx.x, gridDim.x, (uint32_t)p.channels, (uint32_t)p.m_tiles);
    for (uint32_t t = blockIdx.x; bready && t < total && !*abort_flag; t += gridDim.x, ti.next()) {
      const int g = (int)ti.g;
      const TfGroup& G = p.g[g];
      if (!wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.err, kErrTEmpty)) break;
      tc_fence_after();
      if (!wait_bounded(full_bar(stage), phase, abort_flag, p.err, kErrFull)) break;
      tc_fence_after();
      const uint32_t a_src = a_base + stage * p.stage_bytes, b_src = sbase + G.b_off;
      const uint32_t idesc = idesc_bf16(128, G.n_mma, true, true);
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kAccCols);
      for (int k = 0; k < G.kpad / 16; ++k) {
        const uint64_t ad = umma_desc(a_src + k * 2048, G.kpad * 128, 1024, kSwizzle128B);
        const uint64_t bd = umma_desc(b_src + k * 2048, G.kpad * 128, 1024, kSwizzle128B);
        mma_bf16(d_tmem, ad, bd, idesc, k != 0);
      }
      mma_commit(empty_bar(stage));
      mma_commit(tfull_bar(acc));
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    mma_commit(drain_bar);
    wait_drain(drain_bar, 0, p.err, kErrDrain);
  } else if (warp >= 2) {
    // TMEM -> registers -> shared staging tile [rows][128 voxels] -> one TMA store.
    // Two staging buffers; stg_ready (4 warp arrivals) hands a filled buffer to the
    // storing lane, stg_free (1 arrival) returns it once its store has read it.
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;  // which 16-column chunks: 2k + half
    const int xl = q * 32 + lane;  // this thread's voxel within the 128-voxel tile
    int acc = 0;
    uint32_t acc_phase = 0;
    int it = 0;
    TileIter ti;
    ti.init(blockIdx.x, gridDim.x, (uint32_t)p.channels, (uint32_t)p.m_tiles);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x, ++it, ti.next()) {
      const int g = (int)ti.g, c = (int)ti.c, mt = (int)ti.mt;
      const TfGroup& G = p.g[g];
      const int buf = it & 1;
      const uint32_t use_par = (uint32_t)((it >> 1) & 1);
      bool ok = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTFull);
      ok = ok && wait_bounded(stg_free_bar(buf), use_par ^ 1u, abort_flag, p.err, kErrTEmpty);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      // each voxel half holds n_mma rows (a multiple of 16): the stores below need no bounds
      // checks; the TMA store reads only the first n_out rows of each half
      // staging tile [n_mma rows][128 voxels]: one 256-byte (BF16) run per output row
      uint8_t* stg = stg_ptr + (size_t)buf * p.stg_bytes;
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kAccCols);
      if constexpr (!SWZ) {
      // this warp's chunks: c0 = 16 * (2k + half); up to four loads in flight per wait
      for (int k0 = 0; 32 * k0 + 16 * half < G.n_mma; k0 += 4) {
        uint32_t rv[4][16];
        int nld = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c0 = 32 * (k0 + u) + 16 * half;
          if (c0 < G.n_mma) {
            tmem_ld16_nowait(tbase + (uint32_t)c0, rv[u]);
            nld = u + 1;
          }
        }
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c0 = 32 * (k0 + u) + 16 * half;
          if (u < nld) {
            if (OUT_F32) {
              float* dst = reinterpret_cast<float*>(stg) + c0 * 128 + xl;
#pragma unroll
              for (int j = 0; j < 16; ++j) dst[j * 128] = __uint_as_float(rv[u][j]);
            } else {
              __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(stg) + c0 * 128 + xl;
#pragma unroll
              for (int j = 0; j < 16; ++j) dst[j * 128] = __float2bfloat16_rn(__uint_as_float(rv[u][j]));
            }
          }
        }
      }
      } else {
      // BF16: staging halves [voxel half][n_mma rows][64 voxels], 128-byte swizzled (16-byte
      // chunk index XOR row % 8).  16 x 256-bit TMEM loads give each thread two voxels x two
      // adjacent columns; packed to BF16 pairs they are mma fragments, and stmatrix .trans
      // writes each 8 voxel x 8 column block as 8 rows of 16 bytes (conflict-free).
      const uint32_t stg_h = stg_base + (uint32_t)(buf * p.stg_bytes) + (uint32_t)((q >> 1) * G.n_mma * 128);
      const int vq = (q & 1) * 4;  // this warp's first 8-voxel chunk within its half
      const int mm = lane >> 3, rr = lane & 7;  // matrix and row whose address this thread gives
      const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kAccCols);
      for (int k0 = 0; 32 * k0 + 16 * half < G.n_mma; k0 += 2) {
        uint32_t rv[2][2][2][4];  // [chunk][16-lane block][8-column half][regs]
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c0 = 32 * (k0 + u) + 16 * half;
          if (c0 < G.n_mma) {
#pragma unroll
            for (int lb = 0; lb < 2; ++lb)
#pragma unroll
              for (int ch = 0; ch < 2; ++ch)
                tmem_ld_16x256b_nowait(tl + ((uint32_t)(16 * lb) << 16) + (uint32_t)(c0 + 8 * ch), rv[u][lb][ch]);
          }
        }
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c0 = 32 * (k0 + u) + 16 * half;
          if (c0 < G.n_mma) {
#pragma unroll
            for (int lb = 0; lb < 2; ++lb) {
              // matrices: 0 = voxels 0-7 x columns 0-7, 1 = voxels 8-15 x 0-7, 2 = 0-7 x 8-15, 3 = 8-15 x 8-15
              const uint32_t m0 = pack_bf16x2(rv[u][lb][0][0], rv[u][lb][0][1]);
              const uint32_t m1 = pack_bf16x2(rv[u][lb][0][2], rv[u][lb][0][3]);
              const uint32_t m2 = pack_bf16x2(rv[u][lb][1][0], rv[u][lb][1][1]);
              const uint32_t m3 = pack_bf16x2(rv[u][lb][1][2], rv[u][lb][1][3]);
              const int c = c0 + ((mm >> 1) << 3) + rr, vc = vq + 2 * lb + (mm & 1);
              stmatrix_x4_trans(stg_h + (uint32_t)(c * 128 + ((vc ^ (c & 7)) << 4)), m0, m1, m2, m3);
            }
          }
        }
      }
      }
      // accumulator drained: hand it back to the MMA warp; staging filled: hand it to the store
      tc_fence_before();
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(tempty_bar(acc));
        mbar_arrive(stg_ready_bar(buf));
      }
      if (warp == 2) {
        bool lead_ok = true;
        if (lane == 0) {
          lead_ok = wait_bounded(stg_ready_bar(buf), use_par, abort_flag, p.err, kErrTFull);
          if (lead_ok) {
            const uint32_t src = stg_base + (uint32_t)(buf * p.stg_bytes);
            if (!SWZ) {
              tma_store_3d(&p.mapY[g], src, mt * 128, 0, c);  // box {128 voxels, n_out rows, 1}
            } else {  // two swizzled boxes {64 voxels, n_out rows, 1}
              tma_store_3d(&p.mapY[g], src, mt * 128, 0, c);
              tma_store_3d(&p.mapY[g], src + (uint32_t)(G.n_mma * 128), mt * 128 + 64, 0, c);
            }
            bulk_commit();
            // the previous tile's store has finished reading its buffer: release it
            bulk_wait_read<1>();
            if (it >= 1) mbar_arrive(stg_free_bar(buf ^ 1));
          }
        }
        if (!__shfl_sync(0xffffffffu, lead_ok ? 1 : 0, 0)) break;
      }
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    if (warp == 2 && lane == 0) bulk_wait<0>();
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

PFN_cuTensorMapEncodeTiled_v12000 tf_encode() {
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

int tf_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

int tf_major() {
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  return major;
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

constexpr size_t kSmemLimit = 220 * 1024;

}  // namespace

cudaError_t tc_basis_tables_create(const BasisHost& h, TcBasisTables& t, std::string& err) {
  t = TcBasisTables();
  t.n_shells = int(h.shells.size());
  t.N = h.N;
  if (t.n_shells > kMaxTcGroups) return cudaSuccess;  // CUDA-core kernels only
  std::vector<__nv_bfloat16> img;
  for (int s = 0; s < t.n_shells; ++s) {
    const ShellHost& sh = h.shells[s];
    t.m[s] = sh.m;
    t.dir_off[s] = sh.dir_off;
    for (int kind = 0; kind < 4; ++kind) {
      // T[i][j] of this kind and its (n_out, n_in)
      const bool out_is_coef = (kind == 0 || kind == 3);
      const int n_out = out_is_coef ? h.N : sh.m, n_in = out_is_coef ? sh.m : h.N;
      auto T = [&](int i, int j) -> double {
        switch (kind) {
          case 0: return sh.P[size_t(i) * sh.m + j];   // P [N][m]
          case 1: return sh.B[size_t(i) * h.N + j];    // B [m][N]
          case 2: return sh.P[size_t(j) * sh.m + i];   // P^T [m][N]
          default: return sh.B[size_t(j) * h.N + i];   // B^T [N][m]
        }
      };
      const int kpad = round_up(n_in, 16), npad = round_up(n_out, 64);
      t.n_in[s][kind] = n_in;
      t.n_out[s][kind] = n_out;
      t.kpad[s][kind] = kpad;
      t.npad[s][kind] = npad;
      size_t off = (img.size() + 511) / 512 * 512;  // 1 KiB aligned (in elements of 2 bytes)
      img.resize(off + size_t(kpad) * npad, __float2bfloat16_rn(0.f));
      for (int k = 0; k < n_in; ++k)
        for (int n = 0; n < n_out; ++n) img[off + size_t(k) * npad + n] = __float2bfloat16_rn(float(T(n, k)));
      t.off[s][kind] = off * 2;
    }
  }
  cudaError_t e = cudaMalloc(&t.d_mem, img.size() * 2);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return e;
  }
  e = cudaMemcpy(t.d_mem, img.data(), img.size() * 2, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    cudaFree(t.d_mem);
    t.d_mem = nullptr;
    return e;
  }
  t.ok = true;
  return cudaSuccess;
}

void tc_basis_tables_destroy(TcBasisTables& t) {
  if (t.d_mem) cudaFree(t.d_mem);
  t.d_mem = nullptr;
  t.ok = false;
}

bool tc_transform_supported(const TcBasisTables& t, int kind, int64_t ldx, int64_t ldy, int out_t) {
  (void)ldx;
  (void)ldy;
  (void)out_t;
  if (!t.ok || !tc_enabled() || !tf_encode() || tf_major() != 10) return false;
  size_t btot = 0;
  int kmax = 0;
  for (int s = 0; s < t.n_shells; ++s) {
    if (t.n_in[s][kind] > 256 || t.n_out[s][kind] > 256) return false;
    btot += size_t(t.kpad[s][kind]) * t.npad[s][kind] * 2;
    kmax = std::max(kmax, t.kpad[s][kind]);
  }
  int nmax = 0;
  for (int s = 0; s < t.n_shells; ++s) nmax = std::max(nmax, t.n_out[s][kind]);
  const size_t stage = size_t(kmax) * 256;
  const size_t stg = 2 * (size_t(2 * ((nmax + 15) / 16 * 16) * 64 * (out_t == 0 ? 4 : 2)) + 1024);
  return btot + 2 * stage + stg + 4096 <= kSmemLimit;
}

cudaError_t tc_transform_launch(const TcBasisTables& t, int kind, const void* X, void* Y, int64_t n_vox, int C,
                                int64_t ldx, int64_t ldy, int out_t, int* err_word, cudaStream_t st) {
  auto fn = tf_encode();
  if (!fn) return cudaErrorNotSupported;
  static const char* kNames[4] = {"signal2sh_tc", "sh2signal_tc", "signal2sh_bwd_tc", "sh2signal_bwd_tc"};
  TraceScope trace(kNames[kind & 3], st);
  TfParams p;
  memset(&p, 0, sizeof p);
  const bool x_is_sig = (kind == 0 || kind == 3);  // input rows in the signal layout
  uint32_t boff = 0;
  int kmax = 0;
  for (int s = 0; s < t.n_shells; ++s) {
    const int n_in = t.n_in[s][kind], n_out = t.n_out[s][kind];
    const int kpad = t.kpad[s][kind], npad = t.npad[s][kind];
    const int64_t sig_row0 = int64_t(C) * t.dir_off[s], sig_cs = t.m[s];
    const int64_t sh_row0 = int64_t(s) * C * t.N, sh_cs = t.N;
    const int64_t x_row0 = x_is_sig ? sig_row0 : sh_row0, x_cs = x_is_sig ? sig_cs : sh_cs;
    TfGroup& G = p.g[s];
    G.y_row0 = x_is_sig ? sh_row0 : sig_row0;
    G.y_cstride = x_is_sig ? sh_cs : sig_cs;
    G.n_out = n_out;
    G.n_mma = round_up(n_out, 16);
    G.kpad = kpad;
    G.npad = npad;
    G.b_off = boff;
    boff += uint32_t(kpad) * npad * 2;
    kmax = std::max(kmax, kpad);
    // A: 3-D {voxels, rows of one channel, channels}
    {
      const char* base = static_cast<const char*>(X) + x_row0 * ldx * 2;
      cuuint64_t dims[3] = {(cuuint64_t)n_vox, (cuuint64_t)n_in, (cuuint64_t)C};
      cuuint64_t strides[2] = {(cuuint64_t)ldx * 2, (cuuint64_t)(x_cs * ldx * 2)};
      cuuint32_t box[3] = {64, (cuuint32_t)kpad, 1};
      cuuint32_t es[3] = {1, 1, 1};
      if (fn(&p.mapA[s], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<char*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
    // B: 2-D {npad columns, kpad rows} of this group's image
    {
      const char* base = static_cast<const char*>(t.d_mem) + t.off[s][kind];
      cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)kpad};
      cuuint64_t strides[1] = {(cuuint64_t)npad * 2};
      cuuint32_t box[2] = {64, (cuuint32_t)kpad};
      cuuint32_t es[2] = {1, 1};
      if (fn(&p.mapB[s], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<char*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
  }
  // output maps.  BF16 outputs of 64 or more rows (SH2Signal and the Signal2SH adjoint at
  // order 8) go through the stmatrix epilogue: measured 0.62 -> 0.50 ms and 0.164 ->
  // 0.135 ms; the 45-row coefficient outputs stay faster with one 128-voxel box
  const int es = out_t == 0 ? 4 : 2;
  int nmax = 0;
  for (int s = 0; s < t.n_shells; ++s) nmax = std::max(nmax, p.g[s].n_out);
  p.swz = (out_t != 0 && nmax >= 64) ? 1 : 0;
  for (int s = 0; s < t.n_shells; ++s) {
    const TfGroup& G = p.g[s];
    const char* base = static_cast<const char*>(Y) + G.y_row0 * ldy * es;
    cuuint64_t dims[3] = {(cuuint64_t)n_vox, (cuuint64_t)G.n_out, (cuuint64_t)C};
    cuuint64_t strides[2] = {(cuuint64_t)ldy * es, (cuuint64_t)(G.y_cstride * ldy * es)};
    // FP32: one box of 128 voxels, staging unswizzled; BF16: boxes of 64 voxels (128-byte rows)
    // read from the 128-byte-swizzled staging halves
    cuuint32_t box[3] = {p.swz ? 64u : 128u, (cuuint32_t)G.n_out, 1};
    cuuint32_t esz[3] = {1, 1, 1};
    if (fn(&p.mapY[s], out_t == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
           const_cast<char*>(base), dims, strides, box, esz, CU_TENSOR_MAP_INTERLEAVE_NONE,
           p.swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  p.n_groups = t.n_shells;
  p.channels = C;
  p.m_tiles = (int)((n_vox + 127) / 128);
  p.stage_bytes = kmax * 256;
  const int nmma_max = (nmax + 15) / 16 * 16;  // nmax: widest group output (above)
  p.stg_bytes = (2 * nmma_max * 64 * es + 1023) / 1024 * 1024;
  p.b_total = (boff + 1023) / 1024 * 1024;
  const size_t fixed = 1024 + p.b_total + 2 * (size_t)p.stg_bytes + 16 * 8 + 128;
  int stages = (int)((kSmemLimit - fixed) / p.stage_bytes);
  stages = std::max(2, std::min(8, stages));
  p.stages = stages;
  p.total_tiles = (int64_t)t.n_shells * C * p.m_tiles;
  if (p.total_tiles >= (int64_t(1) << 31)) return cudaErrorInvalidValue;  // the kernel walks tiles in 32 bits
  p.n_vox = n_vox;
  p.ldy = ldy;
  p.Y = Y;
  p.err = err_word;
  // at least 120 KiB so that two CTAs never share an SM (each holds 512 TMEM columns)
  const size_t smem = std::max<size_t>(120 * 1024, fixed + (size_t)stages * p.stage_bytes + (2 * stages + 10) * 8);
  if (p.total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(p.total_tiles, tf_sms());
  cudaError_t e;
  auto kern = out_t == 0 ? transform_tc_kernel<true, false>
                         : (p.swz ? transform_tc_kernel<false, true> : transform_tc_kernel<false, false>);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, st>>>(p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace delimit
