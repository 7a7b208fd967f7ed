// tcgen05 + TMA GEMMs of the LSC's BF16 path (collapsed operator, Sec. 2.3).
//
// Activations are feature-rows x voxel-columns with voxels contiguous (the
// paper's tensor convention, Sec. 2.1), so every TMA box is 64 voxels (128 B,
// 128-byte swizzle) wide and feature rows (any count, e.g. 45 coefficients)
// never meet an alignment rule.
//
//   vox_gemm   forward and input-gradient: D[voxel, feature] in TMEM,
//              A = activations (MN-major), B = collapsed operator (MN-major)
//   wgrad      weight gradient: D[out feature, in feature], both operands
//              K-major (voxels are the reduction), voxel range split for occupancy
//
// CTA layout (192 threads): warp 0 issues TMA, warp 1 owns TMEM and issues
// MMAs (one lane), warps 2-5 drain TMEM (each its 32-lane quarter).  Shared
// memory holds a ring of STAGES operand stages; TMEM holds two accumulators so
// the epilogue of one tile overlaps the MMAs of the next.  Every mbarrier wait
// is bounded (ptx::kWaitLimitNs); on expiry the kernel records an error code,
// waits (bounded) for its own copies and MMAs in flight, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <mutex>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace delimit {

namespace {

std::atomic<bool> g_tc_on{true};

enum : int {
  kErrFull = 0x100,
  kErrEmpty = 0x200,
  kErrTmemFull = 0x300,
  kErrTmemEmpty = 0x400,
  kErrDrain = 0x500,
};

constexpr int kEpiWarps = 8;                 // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // + TMA warp + MMA warp
constexpr int kBK = 64;            // K rows (or voxels) per stage
constexpr int kBoxBytes = 64 * 128;  // one 64 x 64 BF16 box, 128-byte rows

}  // namespace

void tc_set_enabled(bool on) { g_tc_on.store(on); }
bool tc_enabled() { return g_tc_on.load(); }

// ---------------------------------------------------------------------------
// forward / input-gradient GEMM
// ---------------------------------------------------------------------------
struct VoxGroup {
  int a_k0, K;      // first K row of both operands, K extent
  int b_n0, N;      // first operator column (multiple of 8), valid output columns
  int64_t y_row0;   // first output row
  int n_tiles;
};

struct VoxParams {
  VoxGroup g[kMaxGroups];
  int n_groups, m_tiles, tiles_per_m;
  int64_t total_tiles, n_vox, ldy;
  __nv_bfloat16* Y;
  const float* bias;
  int* err;
};

__device__ __forceinline__ void vox_decode(const VoxParams& p, int64_t t, int& g, int& mt, int& nt) {
  mt = (int)(t / p.tiles_per_m);
  int r = (int)(t % p.tiles_per_m);
  g = 0;
  while (r >= p.g[g].n_tiles) {
    r -= p.g[g].n_tiles;
    ++g;
  }
  nt = r;
}

// STAGED: the epilogue writes the tile to shared memory and stores it with TMA
// through mapY (3-D {voxels, N rows of a group, groups}: rows past a group's N
// are clipped); otherwise each lane stores its voxel's columns directly.
template <int BN, int STAGES, bool STAGED>
__global__ void __launch_bounds__(kThreads, 1)
    vox_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const __grid_constant__ CUtensorMap mapY, const __grid_constant__ VoxParams p) {
  using namespace ptx;
  constexpr int A_BYTES = 2 * kBoxBytes;        // 128 voxels x 64 K rows
  constexpr int B_BYTES = (BN / 64) * kBoxBytes;  // BN columns x 64 K rows
  constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int HB = BN / 2;                             // columns per staged pass
  constexpr int STG_BYTES = STAGED ? HB * 128 * 2 : 0;  // [HB rows][64 voxels] x 2 voxel halves, BF16
  constexpr uint32_t TMEM_COLS = (2 * BN <= 256) ? 256 : 512;
  constexpr uint32_t IDESC = idesc_bf16(128, BN, true, true);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stg_ptr = smem + STAGES * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_ptr + STG_BYTES);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain, stg_ready, stg_free
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 7);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t sbase = smem_u32(smem);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto tfull_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };
  const uint32_t drain_bar = smem_u32(bars + 2 * STAGES + 4);
  const uint32_t stg_ready_bar = smem_u32(bars + 2 * STAGES + 5);
  const uint32_t stg_free_bar = smem_u32(bars + 2 * STAGES + 6);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    mbar_init(stg_ready_bar, kEpiWarps);
    mbar_init(stg_free_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
    if (STAGED) prefetch_tmap(&mapY);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int stage = 0;
    uint32_t phase = 0;
    int pend[STAGES];
    for (int s = 0; s < STAGES; ++s) pend[s] = -1;
    for (int64_t t = blockIdx.x; t < p.total_tiles && !*abort_flag; t += gridDim.x) {
      int g, mt, nt;
      vox_decode(p, t, g, mt, nt);
      const VoxGroup& G = p.g[g];
      const int nkb = (G.K + kBK - 1) / kBK;
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, p.err, kErrEmpty)) {
          ok = false;
          break;
        }
        const uint32_t a_dst = sbase + stage * STAGE_BYTES, b_dst = a_dst + A_BYTES;
        mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
        const int krow = G.a_k0 + kb * kBK;
        tma_load_2d(&mapA, full_bar(stage), a_dst, mt * 128, krow);
        tma_load_2d(&mapA, full_bar(stage), a_dst + kBoxBytes, mt * 128 + 64, krow);
#pragma unroll
        for (int j = 0; j < BN / 64; ++j)
          tma_load_2d(&mapB, full_bar(stage), b_dst + j * kBoxBytes, G.b_n0 + nt * BN + j * 64, krow);
        pend[stage] = (int)phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
    }
    // copies still in flight complete before the CTA may exit
    for (int s = 0; s < STAGES; ++s)
      if (pend[s] >= 0) wait_drain(full_bar(s), (uint32_t)pend[s], p.err, kErrDrain);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int64_t t = blockIdx.x; t < p.total_tiles && !*abort_flag; t += gridDim.x) {
      int g, mt, nt;
      vox_decode(p, t, g, mt, nt);
      const int nkb = (p.g[g].K + kBK - 1) / kBK;
      if (!wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.err, kErrTmemEmpty)) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!wait_bounded(full_bar(stage), phase, abort_flag, p.err, kErrFull)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_src = sbase + stage * STAGE_BYTES, b_src = a_src + A_BYTES;
#pragma unroll
        for (int k = 0; k < kBK / 16; ++k) {
          // MN-major, 128-byte swizzle: 64-element MN atoms kBoxBytes apart (LBO),
          // 8-row K groups 1024 B apart (SBO); 16 K rows = 2048 B per MMA.
          const uint64_t ad = umma_desc(a_src + k * 2048, kBoxBytes, 1024, kSwizzle128B);
          const uint64_t bd = umma_desc(b_src + k * 2048, kBoxBytes, 1024, kSwizzle128B);
          mma_bf16(d_tmem, ad, bd, IDESC, (kb | k) != 0);
        }
        mma_commit(empty_bar(stage));
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(tfull_bar(acc));
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    mma_commit(drain_bar);
    wait_drain(drain_bar, 0, p.err, kErrDrain);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // 16-column chunks 2k + half
    int acc = 0;
    uint32_t acc_phase = 0;
    int it = 0;
    const int h = q >> 1, xl = (q & 1) * 32 + lane;
    for (int64_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x, ++it) {
      int g, mt, nt;
      vox_decode(p, t, g, mt, nt);
      const VoxGroup& G = p.g[g];
      bool ok = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTmemFull);
      if (STAGED) ok = ok && wait_bounded(stg_free_bar, (uint32_t)((2 * it) & 1) ^ 1u, abort_flag, p.err, kErrTmemEmpty);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int64_t vox = (int64_t)mt * 128 + q * 32 + lane;
      const bool vok = vox < p.n_vox;
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
      if (STAGED) {
        // two passes of HB columns through one staging tile, each stored by TMA
        bool alive = true;
        for (int pass = 0; pass < 2 && alive; ++pass) {
          const int use = 2 * it + pass;
          if (pass == 1) {
            bool okf = wait_bounded(stg_free_bar, (uint32_t)(use & 1) ^ 1u, abort_flag, p.err, kErrTmemEmpty);
            if (!__all_sync(0xffffffffu, okf)) {
              alive = false;
              break;
            }
          }
          const int cbeg = pass * HB;
          for (int k0 = 0; 32 * k0 + 16 * half < HB; k0 += 4) {
            uint32_t rv[4][16];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c0 = cbeg + 32 * (k0 + u) + 16 * half;
              if (c0 < cbeg + HB) tmem_ld16_nowait(tbase + (uint32_t)c0, rv[u]);
            }
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c0 = cbeg + 32 * (k0 + u) + 16 * half;
              const int nbase = nt * BN + c0;
              if (c0 < cbeg + HB) {
                __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(stg_ptr) + (size_t)h * HB * 64 + (c0 - cbeg) * 64 + xl;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                  const float bv = (p.bias && nbase + jj < G.N) ? __ldg(p.bias + G.y_row0 + nbase + jj) : 0.f;
                  dst[jj * 64] = __float2bfloat16_rn(__uint_as_float(rv[u][jj]) + bv);
                }
              }
            }
          }
          if (pass == 1) tc_fence_before();
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            if (pass == 1) mbar_arrive(tempty_bar(acc));
            mbar_arrive(stg_ready_bar);
          }
          if (warp == 2) {
            bool lead_ok = true;
            if (lane == 0) {
              lead_ok = wait_bounded(stg_ready_bar, (uint32_t)(use & 1), abort_flag, p.err, kErrTmemFull);
              if (lead_ok) {
                const uint32_t src = smem_u32(stg_ptr);
                tma_store_3d(&mapY, src, mt * 128, nt * BN + cbeg, g);
                tma_store_3d(&mapY, src + HB * 128, mt * 128 + 64, nt * BN + cbeg, g);
                bulk_commit();
                bulk_wait_read<0>();
                mbar_arrive(stg_free_bar);
              }
            }
            if (!__shfl_sync(0xffffffffu, lead_ok ? 1 : 0, 0)) alive = false;
          }
        }
        if (!alive) break;
      } else {
        for (int k0 = 0; 32 * k0 + 16 * half < BN && nt * BN + 32 * k0 + 16 * half < G.N; k0 += 4) {
          uint32_t rv[4][16];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c0 = 32 * (k0 + u) + 16 * half;
            if (c0 < BN && nt * BN + c0 < G.N) tmem_ld16_nowait(tbase + (uint32_t)c0, rv[u]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c0 = 32 * (k0 + u) + 16 * half;
            const int nbase = nt * BN + c0;
            if (c0 < BN && nbase < G.N) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int n = nbase + jj;
                if (n < G.N && vok) {
                  const float bv = p.bias ? __ldg(p.bias + G.y_row0 + n) : 0.f;
                  p.Y[(G.y_row0 + n) * p.ldy + vox] = __float2bfloat16_rn(__uint_as_float(rv[u][jj]) + bv);
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(acc));
      }
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    if (STAGED && warp == 2 && lane == 0) bulk_wait<0>();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// weight-gradient GEMM
// ---------------------------------------------------------------------------
struct WgGroup {
  int64_t m_row0, x_row0, n_col0;
  int M, N, m_tiles, n_tiles;
};

struct WgParams {
  WgGroup g[kMaxGroups];
  int n_groups, splits;
  int64_t tiles_per_split, total_tiles, vps, n_vox, ldp, split_stride;
  float* P;
  int* err;
};

__device__ __forceinline__ void wg_decode(const WgParams& p, int64_t t, int& split, int& g, int& mt, int& nt) {
  split = (int)(t / p.tiles_per_split);
  int64_t r = t % p.tiles_per_split;
  g = 0;
  while (r >= (int64_t)p.g[g].m_tiles * p.g[g].n_tiles) {
    r -= (int64_t)p.g[g].m_tiles * p.g[g].n_tiles;
    ++g;
  }
  mt = (int)(r / p.g[g].n_tiles);
  nt = (int)(r % p.g[g].n_tiles);
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    wgrad_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const __grid_constant__ WgParams p) {
  using namespace ptx;
  constexpr int A_BYTES = 128 * 128;  // 128 rows x 64 voxels
  constexpr int B_BYTES = BN * 128;   // BN rows x 64 voxels
  constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t TMEM_COLS = (2 * BN <= 256) ? 256 : 512;
  constexpr uint32_t IDESC = idesc_bf16(128, BN, false, false);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t sbase = smem_u32(smem);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto tfull_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };
  const uint32_t drain_bar = smem_u32(bars + 2 * STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int stage = 0;
    uint32_t phase = 0;
    int pend[STAGES];
    for (int s = 0; s < STAGES; ++s) pend[s] = -1;
    for (int64_t t = blockIdx.x; t < p.total_tiles && !*abort_flag; t += gridDim.x) {
      int split, g, mt, nt;
      wg_decode(p, t, split, g, mt, nt);
      const WgGroup& G = p.g[g];
      const int64_t vs = (int64_t)split * p.vps, ve = min(p.n_vox, vs + p.vps);
      const int nkb = (int)((ve - vs + 63) / 64);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, p.err, kErrEmpty)) {
          ok = false;
          break;
        }
        const uint32_t a_dst = sbase + stage * STAGE_BYTES, b_dst = a_dst + A_BYTES;
        mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
        const int vx = (int)(vs + (int64_t)kb * 64);
        tma_load_2d(&mapA, full_bar(stage), a_dst, vx, (int)(G.m_row0 + (int64_t)mt * 128));
        tma_load_2d(&mapB, full_bar(stage), b_dst, vx, (int)(G.x_row0 + (int64_t)nt * BN));
        pend[stage] = (int)phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
    }
    for (int s = 0; s < STAGES; ++s)
      if (pend[s] >= 0) wait_drain(full_bar(s), (uint32_t)pend[s], p.err, kErrDrain);
  } else if (warp == 1 && lane == 0) {
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int64_t t = blockIdx.x; t < p.total_tiles && !*abort_flag; t += gridDim.x) {
      int split, g, mt, nt;
      wg_decode(p, t, split, g, mt, nt);
      const int64_t vs = (int64_t)split * p.vps, ve = min(p.n_vox, vs + p.vps);
      const int nkb = (int)((ve - vs + 63) / 64);
      if (!wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.err, kErrTmemEmpty)) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!wait_bounded(full_bar(stage), phase, abort_flag, p.err, kErrFull)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_src = sbase + stage * STAGE_BYTES, b_src = a_src + A_BYTES;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // K-major, 128-byte swizzle: rows 128 B apart, 8-row groups 1024 B apart (SBO);
          // 16 voxels = 32 B per MMA inside the swizzle atom.
          const uint64_t ad = umma_desc(a_src + k * 32, 16, 1024, kSwizzle128B);
          const uint64_t bd = umma_desc(b_src + k * 32, 16, 1024, kSwizzle128B);
          mma_bf16(d_tmem, ad, bd, IDESC, (kb | k) != 0);
        }
        mma_commit(empty_bar(stage));
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(tfull_bar(acc));
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    mma_commit(drain_bar);
    wait_drain(drain_bar, 0, p.err, kErrDrain);
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;  // 16-column chunks 2k + half
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int64_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
      int split, g, mt, nt;
      wg_decode(p, t, split, g, mt, nt);
      const WgGroup& G = p.g[g];
      bool ok = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTmemFull);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
      const int m = mt * 128 + q * 32 + lane;
      float* prow = p.P + (int64_t)split * p.split_stride + (G.m_row0 + m) * p.ldp + G.n_col0;
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
      for (int k0 = 0; 32 * k0 + 16 * half < BN && nt * BN + 32 * k0 + 16 * half < G.N; k0 += 4) {
        uint32_t rv[4][16];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c0 = 32 * (k0 + u) + 16 * half;
          if (c0 < BN && nt * BN + c0 < G.N) tmem_ld16_nowait(tbase + (uint32_t)c0, rv[u]);
        }
        tmem_wait_ld();
        if (m < G.M) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int nbase = nt * BN + 32 * (k0 + u) + 16 * half;
            if (32 * (k0 + u) + 16 * half < BN && nbase < G.N) {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (nbase + j < G.N) prow[nbase + j] = __uint_as_float(rv[u][j]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(acc));
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// Row sums of dY per voxel split (the bias-gradient column of the weight gradient).
__global__ void __launch_bounds__(256) rowsum_kernel(const __nv_bfloat16* __restrict__ dY, int64_t lddy, int64_t rows,
                                                     int64_t n_vox, int64_t vps, int splits, float* __restrict__ P,
                                                     int64_t ldp, int64_t split_stride, int64_t col) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (wid >= rows * splits) return;
  const int64_t row = wid / splits;
  const int split = (int)(wid % splits);
  const int64_t vs = (int64_t)split * vps, ve = min(n_vox, vs + vps);
  const __nv_bfloat16* r = dY + row * lddy;
  float acc = 0.f;
  // vs is a multiple of 128 and rows are 16-byte aligned: 8-element vectors up to the last full one
  const int64_t vend8 = vs + ((ve - vs) / 8) * 8;
  for (int64_t v = vs + (int64_t)lane * 8; v < vend8; v += 256) {
    const uint4 u = *reinterpret_cast<const uint4*>(r + v);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(h[i]);
      acc += f.x + f.y;
    }
  }
  for (int64_t v = vend8 + lane; v < ve; v += 32) acc += __bfloat162float(r[v]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) P[(int64_t)split * split_stride + row * ldp + col] = acc;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

struct DevInfo {
  int sms = 0, major = 0, minor = 0;
};

DevInfo dev_info() {
  static DevInfo cache[128];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 128) return DevInfo{};
  if (cache[dev].sms == 0) {
    cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cache[dev].major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&cache[dev].minor, cudaDevAttrComputeCapabilityMinor, dev);
  }
  return cache[dev];
}

// 2-D BF16 map over a [outer][ld] row-major array using `inner` columns, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld_elems, uint32_t box_inner,
              uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld_elems * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, bool STAGED>
constexpr int vox_stages() {
  // operand ring + (staged) one BN x 128 BF16 output tile within ~210 KiB
  return STAGED ? (BN == 256 ? 4 : (BN == 192 ? 5 : 6)) : ((BN == 256) ? 4 : (BN == 192 ? 5 : 6));
}

template <int BN, int STAGES>
constexpr size_t smem_bytes(int a_bytes, int b_bytes) {
  return 1024 + (size_t)STAGES * (a_bytes + b_bytes) + (2 * STAGES + 5) * 8 + 16;
}

template <int BN, bool STAGED>
cudaError_t launch_vox(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& my, const VoxParams& p,
                       cudaStream_t st) {
  constexpr int S = vox_stages<BN, STAGED>();
  const size_t smem = smem_bytes<BN, S>(2 * kBoxBytes, (BN / 64) * kBoxBytes) + (STAGED ? BN * 128 : 0) + 16;
  auto kern = vox_gemm_kernel<BN, S, STAGED>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int sms = std::max(1, dev_info().sms);
  const unsigned grid = (unsigned)std::min<int64_t>(p.total_tiles, sms);
  { kern<<<grid, kThreads, smem, st>>>(ma, mb, my, p); count_launch(); }
  return cudaGetLastError();
}

// choose the N tile that wastes the fewest columns over the groups (ties: larger)
int pick_bn(const int* Ns, int n) {
  const int cands[3] = {256, 192, 128};
  int best = 256;
  int64_t best_cols = INT64_MAX;
  for (int c : cands) {
    int64_t cols = 0;
    for (int i = 0; i < n; ++i) cols += (int64_t)((Ns[i] + c - 1) / c) * c;
    if (cols < best_cols) {
      best_cols = cols;
      best = c;
    }
  }
  return best;
}

// The staged epilogue is used when every group has the same N (one 3-D output
// map covers them) and the tile is at most 192 wide (ring + tile fit in smem).
cudaError_t run_vox(const CUtensorMap& ma, const CUtensorMap& mb, VoxParams& p, int bn, bool staged_ok,
                    void* Y, int64_t ldy, cudaStream_t st) {
  p.tiles_per_m = 0;
  bool same_n = true;
  for (int i = 0; i < p.n_groups; ++i) {
    p.g[i].n_tiles = (p.g[i].N + bn - 1) / bn;
    p.tiles_per_m += p.g[i].n_tiles;
    same_n = same_n && p.g[i].N == p.g[0].N && p.g[i].y_row0 == (int64_t)i * p.g[0].N;
  }
  p.total_tiles = (int64_t)p.m_tiles * p.tiles_per_m;
  if (p.total_tiles == 0) return cudaSuccess;
  CUtensorMap my;
  memset(&my, 0, sizeof my);
  bool staged = staged_ok && same_n && bn <= 192;
  if (staged) {
    auto fn = encode_fn();
    cuuint64_t dims[3] = {(cuuint64_t)p.n_vox, (cuuint64_t)p.g[0].N, (cuuint64_t)p.n_groups};
    cuuint64_t strides[2] = {(cuuint64_t)ldy * 2, (cuuint64_t)(p.g[0].N * ldy * 2)};
    cuuint32_t box[3] = {64, (cuuint32_t)(bn / 2), 1};
    cuuint32_t es[3] = {1, 1, 1};
    staged = fn(&my, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Y, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  if (staged) {
    switch (bn) {
      case 192: return launch_vox<192, true>(ma, mb, my, p, st);
      default: return launch_vox<128, true>(ma, mb, my, p, st);
    }
  }
  switch (bn) {
    case 256: return launch_vox<256, false>(ma, mb, my, p, st);
    case 192: return launch_vox<192, false>(ma, mb, my, p, st);
    default: return launch_vox<128, false>(ma, mb, my, p, st);
  }
}

int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return (v && *v) ? atoi(v) : dflt;
}

}  // namespace

bool tc_gemm_supported(const LscDims& d, int64_t n_vox, int64_t ld_in, int64_t ld_out) {
  if (!tc_enabled() || !encode_fn()) return false;
  const DevInfo di = dev_info();
  if (di.major != 10) return false;  // tcgen05 family (sm_100 / sm_103)
  if (n_vox < 1 || n_vox > (int64_t(1) << 31) - 256) return false;
  if (d.rows_in >= (int64_t(1) << 31) || d.rows_out >= (int64_t(1) << 31)) return false;
  (void)ld_in;
  (void)ld_out;
  return true;
}

cudaError_t tc_lsc_forward(const LscDims& d, const void* X, const void* Wt, const float* bias, void* Y, int64_t n_vox,
                           int64_t ldx, int64_t ldy, int* err, cudaStream_t st) {
  TraceScope trace("lsc_fwd_gemm", st);
  CUtensorMap ma, mb;
  if (!make_map(&ma, X, (uint64_t)n_vox, (uint64_t)d.rows_in, (uint64_t)ldx, 64, kBK)) return cudaErrorInvalidValue;
  if (!make_map(&mb, Wt, (uint64_t)d.ldWt, (uint64_t)d.rows_in, (uint64_t)d.ldWt, 64, kBK)) return cudaErrorInvalidValue;
  VoxParams p;
  memset(&p, 0, sizeof p);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  int Ns[kMaxGroups];
  for (int s = 0; s < d.s_out; ++s) {
    VoxGroup& G = p.g[s];
    G.a_k0 = d.win_lo[s] * per_in;
    G.K = (d.win_hi[s] - d.win_lo[s]) * per_in;
    G.b_n0 = (int)(s * d.out_blk);
    G.N = per_out;
    G.y_row0 = (int64_t)s * per_out;
    Ns[s] = G.N;
  }
  p.n_groups = d.s_out;
  p.m_tiles = (int)((n_vox + 127) / 128);
  p.n_vox = n_vox;
  p.ldy = ldy;
  p.Y = reinterpret_cast<__nv_bfloat16*>(Y);
  p.bias = bias;
  p.err = err;
  // forward tiles are short in K and wide in output: stage the epilogue through TMA stores
  int bn = pick_bn(Ns, d.s_out);
  if (bn == 256) bn = ((Ns[0] % 192) == 0) ? 192 : 128;
  bn = env_int("DELIMIT_FWD_BN", bn);
  return run_vox(ma, mb, p, bn, env_int("DELIMIT_FWD_STAGED", 1) != 0, Y, ldy, st);
}

cudaError_t tc_lsc_dgrad(const LscDims& d, const void* dY, const void* W, void* dX, int64_t n_vox, int64_t lddy,
                         int64_t lddx, int* err, cudaStream_t st) {
  TraceScope trace("lsc_dgrad_gemm", st);
  CUtensorMap ma, mb;
  if (!make_map(&ma, dY, (uint64_t)n_vox, (uint64_t)d.rows_out, (uint64_t)lddy, 64, kBK)) return cudaErrorInvalidValue;
  if (!make_map(&mb, W, (uint64_t)d.ldW, (uint64_t)d.rows_out, (uint64_t)d.ldW, 64, kBK)) return cudaErrorInvalidValue;
  VoxParams p;
  memset(&p, 0, sizeof p);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  int Ns[kMaxGroups];
  for (int sp = 0; sp < d.s_in; ++sp) {
    VoxGroup& G = p.g[sp];
    G.a_k0 = d.rwin_lo[sp] * per_out;
    G.K = std::max(0, d.rwin_hi[sp] - d.rwin_lo[sp]) * per_out;
    G.b_n0 = (int)(sp * d.in_blk);
    G.N = per_in;
    G.y_row0 = (int64_t)sp * per_in;
    Ns[sp] = G.N;
  }
  p.n_groups = d.s_in;
  p.m_tiles = (int)((n_vox + 127) / 128);
  p.n_vox = n_vox;
  p.ldy = lddx;
  p.Y = reinterpret_cast<__nv_bfloat16*>(dX);
  p.bias = nullptr;
  p.err = err;
  return run_vox(ma, mb, p, env_int("DELIMIT_DGRAD_BN", pick_bn(Ns, d.s_in)), env_int("DELIMIT_DGRAD_STAGED", 0) != 0,
                 dX, lddx, st);
}

cudaError_t tc_lsc_wgrad(const LscDims& d, const void* dY, const void* X, float* P, int64_t ldp, int64_t split_stride,
                         int splits, int64_t vps, int64_t n_vox, int64_t lddy, int64_t ldx, int* err, cudaStream_t st) {
  constexpr int BN = 256, S = 4;
  CUtensorMap ma, mb;
  if (!make_map(&ma, dY, (uint64_t)n_vox, (uint64_t)d.rows_out, (uint64_t)lddy, 64, 128)) return cudaErrorInvalidValue;
  if (!make_map(&mb, X, (uint64_t)n_vox, (uint64_t)d.rows_in, (uint64_t)ldx, 64, BN)) return cudaErrorInvalidValue;
  if (vps % 64 != 0) return cudaErrorInvalidValue;
  WgParams p;
  memset(&p, 0, sizeof p);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  p.tiles_per_split = 0;
  for (int s = 0; s < d.s_out; ++s) {
    WgGroup& G = p.g[s];
    G.m_row0 = (int64_t)s * per_out;
    G.x_row0 = (int64_t)d.win_lo[s] * per_in;
    G.n_col0 = G.x_row0;
    G.M = per_out;
    G.N = (d.win_hi[s] - d.win_lo[s]) * per_in;
    G.m_tiles = (G.M + 127) / 128;
    G.n_tiles = (G.N + BN - 1) / BN;
    p.tiles_per_split += (int64_t)G.m_tiles * G.n_tiles;
  }
  p.n_groups = d.s_out;
  p.splits = splits;
  p.total_tiles = p.tiles_per_split * splits;
  p.vps = vps;
  p.n_vox = n_vox;
  p.ldp = ldp;
  p.split_stride = split_stride;
  p.P = P;
  p.err = err;
  const size_t smem = smem_bytes<BN, S>(128 * 128, BN * 128);
  auto kern = wgrad_kernel<BN, S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int sms = std::max(1, dev_info().sms);
  if (p.total_tiles > 0) {
    TraceScope trace("lsc_wgrad_gemm", st);
    { kern<<<(unsigned)std::min<int64_t>(p.total_tiles, sms), kThreads, smem, st>>>(ma, mb, p); count_launch(); }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t warps = d.rows_out * splits;
  TraceScope trace_rs("lsc_rowsum", st);
  { rowsum_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(dY), lddy, d.rows_out, n_vox, vps, splits, P, ldp, split_stride, d.rows_in); count_launch(); }
  return cudaGetLastError();
}

}  // namespace delimit
