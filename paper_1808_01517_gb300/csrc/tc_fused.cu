// The LSC forward with SH2Signal fused into its epilogue (Sec. 2.3: the paper's example
// pipes SH -> LSC -> SH2Signal), BF16 activations, FP32 accumulation:
//   c_out[(s,co,:), v] = sum_k W[(s,co,:), k] X[k, v] + bias[(s,co,:)]     (the LSC, collapsed)
//   s_out[(s,co,i), v] = sum_a B_s[i][a] bf16(c_out[(s,co,a), v])          (SH2Signal)
// c_out never leaves the chip: each tile's accumulator is rounded to BF16 exactly where
// the unfused chain stores it, staged in shared memory as the A operand of a second
// 2-SM MMA against B_s, and only s_out is written to HBM.
//
// Tiles: CTA pairs (2-SM MMAs, M = 256 voxels, 128 per CTA) x 192 operator rows = four
// whole channels of one output shell, each in a 48-row slot (N_out <= 48; rows past
// N_out read as zero through a 3-D map {K, N_out, channels} of W, so W needs no padded
// copy).  The main loop is the forward GEMM's (TMA ring, one MMA-issuing thread, TMEM
// double buffer).  The epilogue of a tile runs in two rounds of two channels:
//   1. twelve warps read the accumulator, add the bias, round to BF16 and write each
//      channel's 128 voxels x 48 rows into shared memory in the MN-major 128-byte-swizzled
//      operand layout (stmatrix .trans);
//   2. a dedicated warp of the even CTA issues, per channel, the 2-SM MMA
//      D2[256 voxels, 96] = A2[256, 48] x B_s^T[48, 96] (B_s^T resident, K-major, each
//      CTA 48 of the 96 directions), into accumulator columns already read (the first
//      channel of a round) and a spare 96-column TMEM block (the second);
//   3. the epilogue warps read D2, round to BF16 and store it straight from registers into
//      the s_out rows of that shell and channel (lane = voxel: 64 contiguous bytes per warp
//      and direction row).  Staging these rows in shared memory for TMA stores measured
//      slower: the staging writes and the stores' reads share the SM's shared-memory
//      bandwidth with the main MMAs' operand reads.
// TMEM: 2 x 192 accumulator columns + 96 spare (512 allocated).  Every wait is bounded.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace delimit {

namespace {

constexpr int kBN = 192;        // operator rows per tile: 4 channel slots
constexpr int kSlot = 48;       // rows per channel slot (N_out <= kSlot)
constexpr int kDirs = 96;       // SH2Signal outputs per channel slot (m_s <= kDirs)
constexpr int kK = 64;          // K rows per main stage
constexpr int kFEpi = 12;       // epilogue warps, three per TMEM lane quarter
constexpr int kFThreads = 32 * (3 + kFEpi);  // TMA producer, MMA issuer, SH2Signal MMA issuer, epilogue
constexpr int kAccStride = 192;               // TMEM columns between the two accumulators
constexpr int kSpareCol = 384;                // the spare 96-column D2 block
constexpr uint32_t kABytes = 2 * 64 * 128;                 // 128 voxels x 64 K rows
constexpr uint32_t kBBytes = (kBN / 2) * 128;              // this CTA's 96 operator rows x 64 K
constexpr uint32_t kStage = kABytes + kBBytes;             // 28 KiB
constexpr uint32_t kA2Bytes = 2 * kSlot * 128;             // one channel: 128 voxels x 48 rows
constexpr uint32_t kB2Bytes = (kDirs / 2) * 128;           // one shell's B_s^T half: 48 rows x 64 K
constexpr int kMaxShellsF = 4;

enum : int {
  kErrFull = 0x4100,
  kErrEmpty = 0x4200,
  kErrTFull = 0x4300,
  kErrTEmpty = 0x4400,
  kErrA2 = 0x4500,
  kErrD2 = 0x4600,
  kErrDrain = 0x4800
};

}  // namespace

struct FusedParams {
  int a_k0[kMaxShellsF], K[kMaxShellsF];  // the window's first input row and extent per output shell
  int m_dirs[kMaxShellsF];                // directions of each output shell (<= kDirs)
  int64_t s_row0[kMaxShellsF];            // first s_out row of each output shell (c_out * dir_off)
  int n_groups, c_out, n_out, tiles_per_group, m_pairs, stages;
  int64_t total_tiles, n_vox, lds;
  __nv_bfloat16* S;
  const float* bias;  // [rows_out] (s, co, a), or NULL
  int* err;
};

struct FusedMaps {
  CUtensorMap a;                 // X: 2-D {voxels, rows_in}, box {64, 64}
  CUtensorMap b;                 // W: 3-D {K columns, N_out rows, S_out * c_out channels}, box {64, 48, 2}
  CUtensorMap b2;                // B_s^T images: 2-D {64 (a), S_out * 96 (i)}, box {64, 48}
};

// smem: [ring stages x 28 KiB][A2: 2 channels x 12 KiB][B2: S_out x 6 KiB][barriers]
__host__ __device__ constexpr size_t fused_smem(int stages, int shells) {
  return 1024 + (size_t)stages * kStage + 2 * kA2Bytes + (size_t)shells * kB2Bytes + (2 * stages + 16) * 8 + 16;
}

template <int STAGES>
__global__ void __launch_bounds__(kFThreads, 1)
    lsc_fwd_sh2s_kernel(const __grid_constant__ FusedMaps maps, const __grid_constant__ FusedParams p) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t a2_base = sbase + STAGES * kStage;
  const uint32_t b2_base = a2_base + 2 * kA2Bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * kStage + 2 * kA2Bytes + (size_t)p.n_groups * kB2Bytes);
  // bars: full[S], empty[S], tfull[2], tempty[2], a2_full, d2_full, bload, drain, drain2, bpeer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 16);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto tfull_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };
  const uint32_t a2_full = smem_u32(bars + 2 * STAGES + 4);
  const uint32_t d2_full = smem_u32(bars + 2 * STAGES + 5);
  const uint32_t bload_bar = smem_u32(bars + 2 * STAGES + 6);
  const uint32_t drain_bar = smem_u32(bars + 2 * STAGES + 7);
  const uint32_t drain2_bar = smem_u32(bars + 2 * STAGES + 8);
  const uint32_t bpeer_bar = smem_u32(bars + 2 * STAGES + 9);  // the odd CTA's B_s^T half has landed
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rank = (int)cluster_rank();
  const int64_t t_first = (int64_t)cluster_id_x(), t_step = (int64_t)cluster_count_x();
  const int tiles_per_m = p.n_groups * p.tiles_per_group;
  auto decode = [&](int64_t t, int& g, int& mtp, int& nt) {
    mtp = (int)(t / tiles_per_m);
    const int r = (int)(t - (int64_t)mtp * tiles_per_m);
    g = r / p.tiles_per_group;
    nt = r - g * p.tiles_per_group;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 2 * kFEpi);  // both CTAs' epilogues release the pair's accumulator
    }
    mbar_init(a2_full, 2 * kFEpi);  // both CTAs' epilogues have staged a round's two channels
    mbar_init(d2_full, 1);
    mbar_init(bload_bar, 1);
    mbar_init(drain_bar, 1);
    mbar_init(drain2_bar, 1);
    mbar_init(bpeer_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&maps.a);
    prefetch_tmap(&maps.b);
  }
  cluster_sync();  // the peer's barriers exist before any copy or commit reaches them
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_slot), 512);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    // this CTA's half of every shell's B_s^T image, resident for the whole kernel
    mbar_arrive_expect_tx(bload_bar, (uint32_t)(p.n_groups * kB2Bytes));
    for (int s = 0; s < p.n_groups; ++s)
      tma_load_2d(&maps.b2, bload_bar, b2_base + s * kB2Bytes, 0, s * kDirs + rank * (kDirs / 2));
    if (rank == 1) {
      // the even CTA issues the SH2Signal MMAs, which read this half too: tell it once it is in
      if (wait_bounded(bload_bar, 0, abort_flag, p.err, kErrA2)) mbar_arrive_cluster(mapa_shared(bpeer_bar, 0));
    }
    int stage = 0;
    uint32_t phase = 0;
    int pend[STAGES];
    for (int s = 0; s < STAGES; ++s) pend[s] = -1;
    bool ok = true;
    for (int64_t t = t_first; ok && t < p.total_tiles && !*abort_flag; t += t_step) {
      int g, mtp, nt;
      decode(t, g, mtp, nt);
      const int mt = 2 * mtp + rank;
      const int nkb = (p.K[g] + kK - 1) / kK;
      const int z = g * p.c_out + 4 * nt + 2 * rank;  // this CTA's first channel of the tile
      for (int kb = 0; kb < nkb; ++kb) {
        if (!wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, p.err, kErrEmpty)) {
          ok = false;
          break;
        }
        const uint32_t a_dst = sbase + stage * kStage, b_dst = a_dst + kABytes;
        const int krow = p.a_k0[g] + kb * kK;
        // both CTAs' bytes complete on the even CTA's barrier, which that CTA arms
        const uint32_t fb = mapa_shared(full_bar(stage), 0);
        if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * kStage);
        tma_load_2d_pair(&maps.a, fb, a_dst, mt * 128, krow);
        tma_load_2d_pair(&maps.a, fb, a_dst + kABytes / 2, mt * 128 + 64, krow);
        tma_load_3d_pair(&maps.b, fb, b_dst, krow, 0, z);
        pend[stage] = (int)phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    wait_drain(bload_bar, 0, p.err, kErrDrain);
    if (rank == 0)
      for (int s = 0; s < STAGES; ++s)
        if (pend[s] >= 0) wait_drain(full_bar(s), (uint32_t)pend[s], p.err, kErrDrain);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- main MMA issuer (the even CTA) ----------------
    constexpr uint32_t idesc = idesc_bf16(256, kBN, true, false);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int64_t t = t_first; ok && t < p.total_tiles && !*abort_flag; t += t_step) {
      int g, mtp, nt;
      decode(t, g, mtp, nt);
      const int nkb = (p.K[g] + kK - 1) / kK;
      if (!wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.err, kErrTEmpty)) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kAccStride);
      for (int kb = 0; kb < nkb; ++kb) {
        if (!wait_bounded(full_bar(stage), phase, abort_flag, p.err, kErrFull)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_src = sbase + stage * kStage, b_src = a_src + kABytes;
#pragma unroll
        for (int k = 0; k < kK / 16; ++k) {
          // A: MN-major, 64-voxel atoms 8 KiB apart; B: K-major operator rows, 16 K = 32 bytes
          const uint64_t ad = umma_desc(a_src + k * 2048, kABytes / 2, 1024, kSwizzle128B);
          const uint64_t bd = umma_desc(b_src + k * 32, 16, 1024, kSwizzle128B);
          mma_bf16_pair(d_tmem, ad, bd, idesc, (kb | k) != 0);
        }
        mma_commit_pair_mc(empty_bar(stage), 0x3);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit_pair_mc(tfull_bar(acc), 0x3);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    mma_commit_pair(drain_bar);
    wait_drain(drain_bar, 0, p.err, kErrDrain);
  } else if (warp == 2 && lane == 0 && rank == 0) {
    // ---------------- SH2Signal MMA issuer (the even CTA) ----------------
    // per round, the round's two channels: D2 = A2 (this round's staged c_out) x B_s^T
    constexpr uint32_t idesc2 = idesc_bf16(256, kDirs, true, false);
    bool ok = wait_bounded(bload_bar, 0, abort_flag, p.err, kErrA2);
    ok = ok && wait_bounded(bpeer_bar, 0, abort_flag, p.err, kErrA2);
    int acc = 0;
    uint32_t u = 0;  // round counter
    for (int64_t t = t_first; ok && t < p.total_tiles; t += t_step) {
      int g, mtp, nt;
      decode(t, g, mtp, nt);
      for (int r = 0; r < 2; ++r, ++u) {
        if (!wait_bounded(a2_full, u & 1u, abort_flag, p.err, kErrA2)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // the round's first channel into its own (already read) accumulator columns, the
          // second into the spare block
          const uint32_t d2 = tmem_base + (uint32_t)(h == 0 ? acc * kAccStride + 96 * r : kSpareCol);
#pragma unroll
          for (int k = 0; k < kSlot / 16; ++k) {
            const uint64_t ad = umma_desc(a2_base + h * kA2Bytes + k * 2048, kSlot * 128, 1024, kSwizzle128B);
            const uint64_t bd = umma_desc(b2_base + g * kB2Bytes + k * 32, 16, 1024, kSwizzle128B);
            mma_bf16_pair(d2, ad, bd, idesc2, k != 0);
          }
        }
        mma_commit_pair_mc(d2_full, 0x3);
      }
      acc ^= 1;
    }
    mma_commit_pair(drain2_bar);
    wait_drain(drain2_bar, 0, p.err, kErrDrain);
  } else if (warp >= 3) {
    // ---------------- epilogue (twelve warps per CTA) ----------------
    // quarter q = warp % 4 holds voxels 32q .. 32q + 31; the three warps of a quarter (group
    // 0, 1, 2) take 16-column chunks ck = group (+ 3) of each channel of a round
    const int q = warp & 3, grp = (warp - 3) >> 2;
    const int vq = (q & 1) * 4, mm = lane >> 3, rr = lane & 7;
    const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16);
    // 16 accumulator columns from `col` of this quarter's 32 lanes (16x256b loads: two
    // 16-lane blocks x two 8-column halves), issued without waiting
    auto load16 = [&](uint32_t col, uint32_t (&rv)[2][2][4]) {
#pragma unroll
      for (int lb = 0; lb < 2; ++lb)
#pragma unroll
        for (int c8 = 0; c8 < 2; ++c8)
          tmem_ld_16x256b_nowait(lane_base + ((uint32_t)(16 * lb) << 16) + col + (uint32_t)(8 * c8), rv[lb][c8]);
    };
    // the loaded columns plus b[] (columns 2(l%4) + {0, 1, 8, 9}), packed to BF16 and written by
    // stmatrix .trans as rows row0 .. row0 + 15 of a staging half with 128-byte rows (16-byte
    // chunk XOR row % 8)
    auto store16 = [&](const uint32_t (&rv)[2][2][4], uint32_t half_base, int row0, const float (&b)[4]) {
#pragma unroll
      for (int lb = 0; lb < 2; ++lb) {
        const uint32_t* r0 = rv[lb][0];
        const uint32_t* r1 = rv[lb][1];
        const uint32_t m0 = pack_bf16x2f(__uint_as_float(r0[0]) + b[0], __uint_as_float(r0[1]) + b[1]);
        const uint32_t m1 = pack_bf16x2f(__uint_as_float(r0[2]) + b[0], __uint_as_float(r0[3]) + b[1]);
        const uint32_t m2 = pack_bf16x2f(__uint_as_float(r1[0]) + b[2], __uint_as_float(r1[1]) + b[3]);
        const uint32_t m3 = pack_bf16x2f(__uint_as_float(r1[2]) + b[2], __uint_as_float(r1[3]) + b[3]);
        const int c = row0 + ((mm >> 1) << 3) + rr, vc = vq + 2 * lb + (mm & 1);
        stmatrix_x4_trans(half_base + (uint32_t)(c * 128 + ((vc ^ (c & 7)) << 4)), m0, m1, m2, m3);
      }
    };
    int acc = 0;
    uint32_t acc_phase = 0, u = 0;
    bool alive = true;
    for (int64_t t = t_first; alive && t < p.total_tiles; t += t_step) {
      int g, mtp, nt;
      decode(t, g, mtp, nt);
      const int mt = 2 * mtp + rank;
      bool ok = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTFull);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      for (int r = 0; r < 2; ++r, ++u) {
        // 1. c_out + bias -> BF16 -> A2 of both channels of the round (rows a of the 48-row
        //    slot, voxels MN-major): this warp's chunk ck = grp of each
        {
          uint32_t rv[2][2][2][4];
          float b[2][4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = 2 * r + h, co = 4 * nt + j;
            load16((uint32_t)(acc * kAccStride + kSlot * j + 16 * grp), rv[h]);
            const float* brow = p.bias ? p.bias + ((int64_t)g * p.c_out + co) * p.n_out : nullptr;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int a = 16 * grp + 2 * (lane & 3) + (i & 1) + 8 * (i >> 1);
              b[h][i] = (brow && a < p.n_out) ? __ldg(brow + a) : 0.f;
            }
          }
          tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h)
            store16(rv[h], a2_base + (uint32_t)(h * kA2Bytes) + (uint32_t)((q >> 1) * kSlot * 128), 16 * grp, b[h]);
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(mapa_shared(a2_full, 0));
        // 2. the pair's SH2Signal MMAs of this round
        ok = wait_bounded(d2_full, u & 1u, abort_flag, p.err, kErrD2);
        if (!__all_sync(0xffffffffu, ok)) {
          alive = false;
          break;
        }
        tc_fence_after();
        // 3. D2 -> BF16 -> s_out straight from registers: lane = voxel, a warp writes 64
        //    contiguous bytes per direction row
        {
          const int m = p.m_dirs[g];
          const int64_t v = (int64_t)mt * 128 + q * 32 + lane;
          const bool in = v < p.n_vox;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int co = 4 * nt + 2 * r + h;
            const uint32_t d2 = (uint32_t)(h == 0 ? acc * kAccStride + 96 * r : kSpareCol);
            uint32_t rv[2][16];
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2) tmem_ld16_nowait(lane_base + d2 + (uint32_t)(16 * (grp + 3 * c2)), rv[c2]);
            tmem_wait_ld();
            if (in) {
#pragma unroll
              for (int c2 = 0; c2 < 2; ++c2) {
                const int i0 = 16 * (grp + 3 * c2);
                __nv_bfloat16* y = p.S + (p.s_row0[g] + (int64_t)co * m + i0) * p.lds + v;
#pragma unroll
                for (int j = 0; j < 16; ++j, y += p.lds)
                  if (i0 + j < m) *y = __float2bfloat16_rn(__uint_as_float(rv[c2][j]));
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
      }
      if (!alive) break;
      // the accumulator (and the D2 columns in it) is drained: back to the MMA issuer
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(mapa_shared(tempty_bar(acc), 0));
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair frees its TMEM once both CTAs are done with it; after this point no copy, commit
  // or arrival of either CTA targets the other
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, 512);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 fused_encode() {
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

constexpr int kFusedStages = 4;
static_assert(fused_smem(kFusedStages, kMaxShellsF) <= 227 * 1024, "the fused kernel's shared memory");

bool enc(CUtensorMap* m, int rank, const void* base, const cuuint64_t* dims, const cuuint64_t* strides,
         const cuuint32_t* box) {
  auto fn = fused_encode();
  if (!fn) return false;
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), const_cast<cuuint64_t*>(dims),
            const_cast<cuuint64_t*>(strides), const_cast<cuuint32_t*>(box), es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t fused_tables_create(const BasisHost& ob, FusedTables& f, std::string& err) {
  f = FusedTables();
  const int S = int(ob.shells.size());
  if (S > kMaxShellsF || ob.N > kSlot) return cudaSuccess;  // no fused form for this basis
  for (const auto& sh : ob.shells)
    if (sh.m > kDirs) return cudaSuccess;
  // B_s^T as the K-major operator: [S][96 directions][64 coefficients], zero-padded, BF16
  // (rounded as the SH2Signal operator images are: FP64 -> FP32 -> BF16)
  std::vector<__nv_bfloat16> img(size_t(S) * kDirs * 64, __float2bfloat16_rn(0.f));
  for (int s = 0; s < S; ++s) {
    const ShellHost& sh = ob.shells[s];
    for (int i = 0; i < sh.m; ++i)
      for (int a = 0; a < ob.N; ++a)
        img[(size_t(s) * kDirs + i) * 64 + a] = __float2bfloat16_rn(float(sh.B[size_t(i) * ob.N + a]));
  }
  cudaError_t e = cudaMalloc(&f.d_b2, img.size() * 2);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    f.d_b2 = nullptr;
    return e;
  }
  e = cudaMemcpy(f.d_b2, img.data(), img.size() * 2, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    cudaFree(f.d_b2);
    f.d_b2 = nullptr;
    return e;
  }
  f.shells = S;
  for (int s = 0; s < S; ++s) {
    f.m[s] = ob.shells[s].m;
    f.dir_off[s] = ob.shells[s].dir_off;
  }
  f.ok = true;
  return cudaSuccess;
}

void fused_tables_destroy(FusedTables& f) {
  if (f.d_b2) cudaFree(f.d_b2);
  f.d_b2 = nullptr;
  f.ok = false;
}

const char* tc_lsc_fused_unsupported(const LscDims& d, const FusedTables& f, int64_t n_vox) {
  if (!tc_enabled()) return "tensor cores are switched off";
  if (!fused_encode()) return "no TMA descriptor encoder";
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return "needs a tcgen05 GPU";
  if (!f.ok) return "output basis with more than 4 shells, more than 96 directions in a shell or order above 8";
  if (d.s_out != f.shells) return "geometry and output basis differ in shells";
  if (d.n_out > kSlot) return "more than 48 output coefficients";
  if (d.c_out % 4 != 0) return "c_out must be a multiple of 4";
  if (d.in_blk != (int64_t)d.c_in * d.n_in) return "input blocks carry padding (c_in * N_in not a multiple of 8)";
  if (n_vox < 1 || n_vox > (int64_t(1) << 31) - 256) return "voxel count out of range";
  return nullptr;
}

cudaError_t tc_lsc_forward_sh2signal(const LscDims& d, const FusedTables& f, const void* X, const void* W,
                                     const float* bias, void* S, int64_t n_vox, int64_t ldx, int64_t lds, int* err,
                                     cudaStream_t st) {
  TraceScope trace("lsc_fwd_sh2signal", st);
  FusedMaps maps;
  memset(&maps, 0, sizeof maps);
  FusedParams p;
  memset(&p, 0, sizeof p);
  {  // X: {voxels, rows_in}, box {64, 64}
    const cuuint64_t dims[2] = {(cuuint64_t)n_vox, (cuuint64_t)d.rows_in};
    const cuuint64_t strides[1] = {(cuuint64_t)ldx * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kK};
    if (!enc(&maps.a, 2, X, dims, strides, box)) return cudaErrorInvalidValue;
  }
  {  // W: {K columns, N_out rows, S_out * c_out channels}, box {64, 48, 2}: rows past N_out read as zero
    const cuuint64_t dims[3] = {(cuuint64_t)d.ldW, (cuuint64_t)d.n_out, (cuuint64_t)(d.s_out * d.c_out)};
    const cuuint64_t strides[2] = {(cuuint64_t)d.ldW * 2, (cuuint64_t)d.n_out * d.ldW * 2};
    const cuuint32_t box[3] = {64, (cuuint32_t)kSlot, 2};
    if (!enc(&maps.b, 3, W, dims, strides, box)) return cudaErrorInvalidValue;
  }
  {  // B_s^T images: {64 coefficients, S_out * 96 directions}, box {64, 48}
    const cuuint64_t dims[2] = {64, (cuuint64_t)(f.shells * kDirs)};
    const cuuint64_t strides[1] = {64 * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)(kDirs / 2)};
    if (!enc(&maps.b2, 2, f.d_b2, dims, strides, box)) return cudaErrorInvalidValue;
  }
  const int per_in = d.c_in * d.n_in;
  for (int s = 0; s < d.s_out; ++s) {
    p.a_k0[s] = d.win_lo[s] * per_in;
    p.K[s] = (d.win_hi[s] - d.win_lo[s]) * per_in;
    p.m_dirs[s] = f.m[s];
    p.s_row0[s] = (int64_t)d.c_out * f.dir_off[s];
  }
  p.S = static_cast<__nv_bfloat16*>(S);
  p.lds = lds;
  p.n_groups = d.s_out;
  p.c_out = d.c_out;
  p.n_out = d.n_out;
  p.tiles_per_group = d.c_out / 4;
  p.m_pairs = (int)((n_vox + 255) / 256);
  p.stages = kFusedStages;
  p.total_tiles = (int64_t)p.m_pairs * p.n_groups * p.tiles_per_group;
  p.n_vox = n_vox;
  p.bias = bias;
  p.err = err;
  if (p.total_tiles == 0) return cudaSuccess;
  auto kern = lsc_fwd_sh2s_kernel<kFusedStages>;
  const size_t smem = fused_smem(kFusedStages, d.s_out);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static int clusters_cached[128] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kFThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = (dev >= 0 && dev < 128) ? clusters_cached[dev] : 0;
  if (clusters == 0) {
    cfg.gridDim = dim3(2 * 64);
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      return cudaErrorInvalidConfiguration;
    }
    if (dev >= 0 && dev < 128) clusters_cached[dev] = clusters;
  }
  cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(p.total_tiles, clusters)));
  e = cudaLaunchKernelEx(&cfg, kern, maps, p);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace delimit
