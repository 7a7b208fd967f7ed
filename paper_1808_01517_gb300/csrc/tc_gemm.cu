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
#include <utility>
#include <vector>

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
constexpr int kWgradBN = 240;      // weight-gradient column tile (divides 720-multiples: 1440, 2160)
constexpr int kDgradBN = 240;      // input-gradient column tile on Wt (K-major), when it divides c_in n_in
constexpr int kBoxBytes = 64 * 128;  // one 64 x 64 BF16 box, 128-byte rows

}  // namespace

void tc_set_enabled(bool on) { g_tc_on.store(on); }
bool tc_enabled() { return g_tc_on.load(); }

namespace {
// CTAs per cluster of the LSC GEMMs: 0 = each GEMM's default, 1 or 2 forced
// (delimit_set_gemm_cluster).  2 = a CTA pair issuing 2-SM tcgen05 MMAs
// (cta_group::2): each CTA loads its own half of the operands by TMA (no TMA
// multicast anywhere), one thread of the even CTA issues the MMAs for both;
// 1 = single-CTA MMAs (the form shapes that do not split into pairs take).
std::atomic<int> g_gemm_cluster{0};
}  // namespace

void tc_set_gemm_cluster(int cl) { g_gemm_cluster.store(cl); }

// ---------------------------------------------------------------------------
// forward / input-gradient GEMM
// ---------------------------------------------------------------------------
struct VoxGroup {
  int a_k0, K;      // first K row of both operands, K extent
  int b_n0, N;      // first operator column (multiple of 8), valid output columns
  int64_t y_row0;   // first output row
  int n_tiles;
  int bn_last;      // width of the group's last operator tile (<= BN, whole 64-column atoms per CTA)
};

// FP32 operands on the BF16 tensor cores: each operand is stored as three BF16
// parts (x = x0 + x1 + x2 up to 2^-27 |x|, the parts the z planes of its tensor
// map) and a tile accumulates the six part products whose magnitude reaches
// 2^-18 of the leading one; the dropped three stay below 2^-26.  Term t (largest
// first) multiplies part split_part_a(t) of A with part split_part_b(t) of B; the
// kernels issue them smallest first, so the corrections are summed while the
// accumulator is still small.  The TMEM accumulation error grows linearly with the
// number of MMAs added into a running sum (measured: about 3e-8 of the sum per MMA, a
// bias rather than a random walk), so the FP32 path also splits K into chunks of
// chunk_kb blocks: each chunk starts from zero in TMEM and the epilogue adds it to the
// FP32 output (read, add in FP32, write back by the thread that stored the element).
constexpr int kSplitTerms = 6;
// K blocks of 64 per accumulation chunk on the FP32 path.  Measured at 65,536 voxels
// (16 -> 64 channels): relative errors of the forward / input / weight gradient 1.0e-6 /
// 1.1e-6 / 9.7e-7 at 16 blocks (5.4e-7 / 5.8e-7 / 3.7e-7 at 4-8, 1.9e-6 / 2.2e-6 / 1.8e-6 at
// 32); the weight gradient's time 7.18 ms at 16 against 8.16 ms at 4 (more folds).
constexpr int kSplitChunkKb = 16;
__host__ __device__ constexpr int split_part_a(int t) { return t == 2 || t == 3 ? 1 : (t == 5 ? 2 : 0); }
__host__ __device__ constexpr int split_part_b(int t) { return t == 1 || t == 3 ? 1 : (t == 4 ? 2 : 0); }
// accumulation chunks of a K range of nkb blocks (at least one, as the MMA issuer
// commits every tile's accumulator even when it is empty)
__host__ __device__ inline int k_chunks(int nkb, int chunk_kb) { return nkb > 0 ? (nkb + chunk_kb - 1) / chunk_kb : 1; }

struct VoxParams {
  VoxGroup g[kMaxGroups];
  int n_groups, m_tiles, tiles_per_m;
  int b_kmajor;  // operator stored [N rows][K contiguous] (K-major) instead of [K rows][N contiguous]
  int n_terms;   // 1 (BF16 operands) or kSplitTerms (three-part BF16 splits of FP32 operands)
  int chunk_kb;  // K blocks per accumulation chunk (> 0; chunks after the first are added in the epilogue)
  int64_t total_tiles, n_vox, ldy;
  __nv_bfloat16* Y;
  float* Yf;  // FP32 output (direct stores) in place of Y
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

// STAGED: the epilogue writes the tile to shared memory (stmatrix, 128-byte swizzle)
// and its warps copy it out to Y in 16-byte chunks, four 128-byte row segments per
// store instruction (Y 16-byte aligned, ldy a multiple of 8; rows past a group's N
// and voxels past n_vox are skipped); otherwise each lane stores its voxel's
// columns directly.  mapY is unused (kept in the signature the two forms share).
// CL = 2: a cluster of two CTAs computes a 256-voxel x BN tile with 2-SM MMAs
// (M = 256): each CTA stages its own 128 voxels of A and BN/2 of the BN
// operator columns, so a CTA takes in half the operator bytes per FLOP of the
// single-CTA form.  The even CTA arms the stage barriers and issues the MMAs;
// each CTA's TMEM receives its own 128 voxels x BN accumulator, drained by its
// own epilogue, which hands the buffer back on the even CTA's barrier.
// p.total_tiles counts cluster tiles (voxel-tile pairs x operator tiles).
template <int BN, int STAGES, bool STAGED, int PASSES, int CL, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    vox_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const __grid_constant__ CUtensorMap mapY, const __grid_constant__ VoxParams p) {
  using namespace ptx;
  static_assert(CL == 1 || CL == 2, "one CTA or a CTA pair");
  // MN-major operators need whole 64-column atoms per CTA (checked on the host); K-major ones
  // only whole 8-row groups (BN = 240 for the input gradient)
  static_assert((BN / CL) % 8 == 0, "whole 8-row operator groups per CTA");
  static_assert(!STAGED || BN % 64 == 0, "the staged epilogue's bias map covers 64-column atoms");
  static_assert(!(SPLIT && STAGED), "FP32 outputs leave through direct stores");
  // SPLIT: FP32 operands as three BF16 planes (3-D maps), six terms, chunked K, FP32 output
  const int n_terms = SPLIT ? p.n_terms : 1;
  const int chunk_kb = SPLIT ? p.chunk_kb : (1 << 24);
  constexpr int A_BYTES = 2 * kBoxBytes;               // 128 voxels x 64 K rows
  constexpr int B_BYTES = (BN / CL) * 128;  // this CTA's BN/CL operator columns x 64 K (128 bytes each)
  constexpr int ACC_STRIDE = BN <= 128 ? 128 : 256;  // TMEM columns between the two accumulators
  constexpr int NBREG = (BN / 2 + 31) / 32;  // bias registers: a warp's BN/2 columns over 32 lanes
  constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int HB = BN / PASSES;                        // columns per staged pass
  constexpr int STG_BYTES = STAGED ? HB * 128 * 2 : 0;  // [HB rows][64 voxels] x 2 voxel halves, BF16
  constexpr uint32_t TMEM_COLS = (2 * BN <= 256) ? 256 : 512;
  constexpr uint32_t IDESC = idesc_bf16(128 * CL, BN, true, true);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stg_ptr = smem + STAGES * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_ptr + STG_BYTES);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain (two slots spare)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 7);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t sbase = smem_u32(smem);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto tfull_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };
  const uint32_t drain_bar = smem_u32(bars + 2 * STAGES + 4);
  const int rank = CL > 1 ? (int)cluster_rank() : 0;
  const int64_t t_first = CL > 1 ? (int64_t)cluster_id_x() : (int64_t)blockIdx.x;
  const int64_t t_step = CL > 1 ? (int64_t)cluster_count_x() : (int64_t)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), CL * kEpiWarps);  // both CTAs' epilogues release the pair's accumulator
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (CL > 1) cluster_sync();  // the peer's barriers exist before any copy or commit reaches them
  if (warp == 1) {
    if (CL > 1) {
      tmem_alloc_pair(smem_u32(tmem_slot), TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs of a pair) ----------------
    int stage = 0;
    uint32_t phase = 0;
    int pend[STAGES];
    for (int s = 0; s < STAGES; ++s) pend[s] = -1;
    for (int64_t t = t_first; t < p.total_tiles && !*abort_flag; t += t_step) {
      int g, mt, nt;
      vox_decode(p, t, g, mt, nt);
      mt = mt * CL + rank;
      const VoxGroup& G = p.g[g];
      const int nkb = (G.K + kBK - 1) / kBK;
      const int tile_bn = nt == G.n_tiles - 1 ? G.bn_last : BN;
      // MN-major operator: 64-column boxes of this CTA's tile_bn / CL columns; K-major: one
      // box of BN / CL rows (a narrow tile loads rows it does not use)
      const int nbox = tile_bn / CL / 64;
      const uint32_t bytes = (uint32_t)(A_BYTES + (p.b_kmajor ? B_BYTES : nbox * kBoxBytes));
      const int ncol = G.b_n0 + nt * BN + rank * (tile_bn / CL);
      bool ok = true;
      const int nch = SPLIT ? k_chunks(nkb, chunk_kb) : 1;
      for (int c = 0; c < nch && ok; ++c)
      for (int ti = 0; ti < n_terms && ok; ++ti) {
        const int term = n_terms - 1 - ti;  // smallest part products first
        const int za = split_part_a(term), zb = split_part_b(term);  // operand planes (0 for BF16)
        for (int kb = c * chunk_kb; kb < min(nkb, (c + 1) * chunk_kb); ++kb) {
          if (!wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, p.err, kErrEmpty)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = sbase + stage * STAGE_BYTES, b_dst = a_dst + A_BYTES;
          const int krow = G.a_k0 + kb * kBK;
          // operand tiles: plane z of a split operand (3-D map), or the BF16 array (2-D map)
          auto load = [&](const CUtensorMap* m, uint32_t bar, uint32_t dst, int x, int y, int z) {
            if constexpr (SPLIT) {
              if (CL > 1)
                tma_load_3d_pair(m, bar, dst, x, y, z);
              else
                tma_load_3d(m, bar, dst, x, y, z);
            } else {
              if (CL > 1)
                tma_load_2d_pair(m, bar, dst, x, y);
              else
                tma_load_2d(m, bar, dst, x, y);
            }
          };
          uint32_t fb = full_bar(stage);
          if (CL > 1) {
            // both CTAs' bytes complete on the even CTA's barrier, which that CTA arms
            fb = mapa_shared(full_bar(stage), 0);
            if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), CL * bytes);
          } else {
            mbar_arrive_expect_tx(full_bar(stage), bytes);
          }
          load(&mapA, fb, a_dst, mt * 128, krow, za);
          load(&mapA, fb, a_dst + kBoxBytes, mt * 128 + 64, krow, za);
          if (p.b_kmajor)
            load(&mapB, fb, b_dst, krow, ncol, zb);
          else
            for (int j = 0; j < nbox; ++j) load(&mapB, fb, b_dst + j * kBoxBytes, ncol + j * 64, krow, zb);
          pend[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) break;
    }
    // copies still in flight complete before the CTA may exit (a pair's odd CTA is
    // covered by the even CTA's drain and the closing cluster barrier)
    if (rank == 0)
      for (int s = 0; s < STAGES; ++s)
        if (pend[s] >= 0) wait_drain(full_bar(s), (uint32_t)pend[s], p.err, kErrDrain);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer (the even CTA of a pair) ----------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int64_t t = t_first; ok && t < p.total_tiles && !*abort_flag; t += t_step) {
      int g, mt, nt;
      vox_decode(p, t, g, mt, nt);
      const int nkb = (p.g[g].K + kBK - 1) / kBK;
      const bool bk = p.b_kmajor != 0;
      const uint32_t idesc = idesc_bf16(128 * CL, nt == p.g[g].n_tiles - 1 ? p.g[g].bn_last : BN, true, !bk);
      const int nch = SPLIT ? k_chunks(nkb, chunk_kb) : 1;
      for (int c = 0; c < nch; ++c) {
        if (!wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.err, kErrTmemEmpty)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * ACC_STRIDE);
        // this chunk's K blocks of every term, in the producer's order
        const int nk = SPLIT ? max(0, min(chunk_kb, nkb - c * chunk_kb)) * n_terms : nkb;
        for (int kb = 0; kb < nk; ++kb) {
          if (!wait_bounded(full_bar(stage), phase, abort_flag, p.err, kErrFull)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_src = sbase + stage * STAGE_BYTES, b_src = a_src + A_BYTES;
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            // MN-major, 128-byte swizzle: 64-element MN atoms kBoxBytes apart (LBO),
            // 8-row K groups 1024 B apart (SBO); 16 K rows = 2048 B per MMA.  K-major
            // operator: rows 128 B apart, 8-row groups 1024 B apart, 16 K = 32 B per MMA.
            const uint64_t ad = umma_desc(a_src + k * 2048, kBoxBytes, 1024, kSwizzle128B);
            const uint64_t bd = bk ? umma_desc(b_src + k * 32, 16, 1024, kSwizzle128B)
                                   : umma_desc(b_src + k * 2048, kBoxBytes, 1024, kSwizzle128B);
            if (CL > 1)
              mma_bf16_pair(d_tmem, ad, bd, idesc, (kb | k) != 0);
            else
              mma_bf16(d_tmem, ad, bd, idesc, (kb | k) != 0);
          }
          if (CL > 1)
            mma_commit_pair_mc(empty_bar(stage), 0x3);  // both CTAs' producers refill this stage
          else
            mma_commit(empty_bar(stage));
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (CL > 1)
          mma_commit_pair_mc(tfull_bar(acc), 0x3);
        else
          mma_commit(tfull_bar(acc));
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1u;
      }
    }
    if (CL > 1)
      mma_commit_pair(drain_bar);
    else
      mma_commit(drain_bar);
    wait_drain(drain_bar, 0, p.err, kErrDrain);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // 16-column chunks 2k + half
    int acc = 0;
    uint32_t acc_phase = 0;
    const int h = q >> 1;
    for (int64_t t = t_first; t < p.total_tiles; t += t_step) {
      int g, mt, nt;
      vox_decode(p, t, g, mt, nt);
      mt = mt * CL + rank;
      const VoxGroup& G = p.g[g];
      // bias of this warp's columns, fetched before the accumulator is ready (a load per
      // column inside the drain loop stalled it): lane L holds the warp's columns
      // w = L + 32 i, i.e. chunk w / 16 (tile columns 32 (w / 16) + 16 half + w % 16)
      float breg[NBREG];
#pragma unroll
      for (int i = 0; i < NBREG; ++i) {
        const int w = lane + 32 * i, col = nt * BN + 32 * (w >> 4) + 16 * half + (w & 15);
        breg[i] = (PASSES == 1 && p.bias && col < G.N) ? __ldg(p.bias + G.y_row0 + col) : 0.f;
      }
      bool ok = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTmemFull);
      // the staged form's warps meet at named barriers, so they leave together: one gave up,
      // all do (a bounded wait that ran out in one warp may have just completed in another)
      if (STAGED ? named_bar_any(1, 32 * kEpiWarps, !ok) : !__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int64_t vox = (int64_t)mt * 128 + q * 32 + lane;
      const bool vok = vox < p.n_vox;
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * ACC_STRIDE);
      // accumulator released to the MMA issuer (the even CTA's barrier for a pair)
      const uint32_t tempty = CL > 1 ? mapa_shared(tempty_bar(acc), 0) : tempty_bar(acc);
      if (STAGED) {
        // PASSES passes of HB columns through one staging tile, copied out to Y by the
        // epilogue warps themselves with streaming (evict-first) stores, so that the
        // output passes L2 without displacing the operand tiles other CTAs still read.
        // Measured 1.16-1.18 ms per forward at 65,536 voxels, as with a TMA store of the
        // tile (1.17-1.19); writing the output at all costs about 0.1 ms of it (1.07 ms
        // with the stores left out), by TMA or by the warps alike.
        for (int pass = 0; pass < PASSES; ++pass) {
          const int cbeg = pass * HB;
          // 16 x 256-bit TMEM loads: thread t holds voxels t/4 and t/4 + 8 of a 16-lane block
          // and columns 2(t%4), 2(t%4)+1 (+8); with the bias added and packed to BF16 pairs
          // they are mma fragments, stored by stmatrix .trans into the staging halves
          // [voxel half][HB rows][64 voxels], 128-byte swizzled (16-byte chunk ^ row % 8)
          const uint32_t stg_h = smem_u32(stg_ptr) + (uint32_t)(h * HB * 128);
          const int vq = (q & 1) * 4, mm = lane >> 3, rr = lane & 7;
#pragma unroll
          for (int k0 = 0; k0 < (HB + 31) / 32; k0 += 2) {
            uint32_t rv[2][2][2][4];  // [chunk][16-lane block][8-column half][regs]
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int c0 = cbeg + 32 * (k0 + u) + 16 * half;
              if (c0 < cbeg + HB) {
#pragma unroll
                for (int lb = 0; lb < 2; ++lb)
#pragma unroll
                  for (int ch = 0; ch < 2; ++ch)
                    tmem_ld_16x256b_nowait(tbase + ((uint32_t)(16 * lb) << 16) + (uint32_t)(c0 + 8 * ch), rv[u][lb][ch]);
              }
            }
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int c0 = cbeg + 32 * (k0 + u) + 16 * half;
              if (c0 < cbeg + HB) {
                const int m = k0 + u;  // this warp's chunk number: columns w = 16 m + j of breg's map
                float b[4];            // columns 2(t%4) + {0, 1, 8, 9} of the chunk
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const int jc = 2 * (lane & 3) + (i & 1) + 8 * (i >> 1);
                  if (PASSES == 1)
                    b[i] = __shfl_sync(0xffffffffu, breg[(m >> 1) < NBREG ? (m >> 1) : 0], ((m & 1) * 16 + jc) & 31);
                  else
                    b[i] = (p.bias && nt * BN + c0 + jc < G.N) ? __ldg(p.bias + G.y_row0 + nt * BN + c0 + jc) : 0.f;
                }
#pragma unroll
                for (int lb = 0; lb < 2; ++lb) {
                  const uint32_t* r0 = rv[u][lb][0];
                  const uint32_t* r1 = rv[u][lb][1];
                  const uint32_t m0 = pack_bf16x2f(__uint_as_float(r0[0]) + b[0], __uint_as_float(r0[1]) + b[1]);
                  const uint32_t m1 = pack_bf16x2f(__uint_as_float(r0[2]) + b[0], __uint_as_float(r0[3]) + b[1]);
                  const uint32_t m2 = pack_bf16x2f(__uint_as_float(r1[0]) + b[2], __uint_as_float(r1[1]) + b[3]);
                  const uint32_t m3 = pack_bf16x2f(__uint_as_float(r1[2]) + b[2], __uint_as_float(r1[3]) + b[3]);
                  const int c = (c0 - cbeg) + ((mm >> 1) << 3) + rr, vc = vq + 2 * lb + (mm & 1);
                  stmatrix_x4_trans(stg_h + (uint32_t)(c * 128 + ((vc ^ (c & 7)) << 4)), m0, m1, m2, m3);
                }
              }
            }
          }
          if (pass == PASSES - 1) {
            // the accumulator is read: back to the MMA issuer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (CL > 1)
                mbar_arrive_cluster(tempty);
              else
                mbar_arrive(tempty);
            }
          }
          named_bar(1, 32 * kEpiWarps);  // the staging tile is complete
          // copy-out: 16-byte chunks (8 voxels) of the tile, a warp per 4 rows x 8 chunks, i.e.
          // four 128-byte row segments of Y per store instruction (conflict-free 128-bit
          // shared loads); rows past the group's N and voxels past n_vox are not written
          {
            const int et = threadIdx.x - 64;
#pragma unroll 4
            for (int e = 0; e < 2 * HB * 8 / (32 * kEpiWarps); ++e) {
              const int i = et + 32 * kEpiWarps * e, j = i & 7, rowh = i >> 3;
              const int hh = rowh >= HB ? 1 : 0, c = rowh - hh * HB;
              const int col = nt * BN + cbeg + c;
              const int64_t v0 = (int64_t)mt * 128 + 64 * hh + 8 * j;
              if (col >= G.N || v0 >= p.n_vox) continue;
              const uint4 val =
                  *reinterpret_cast<const uint4*>(stg_ptr + (hh * HB + c) * 128 + ((j ^ (c & 7)) << 4));
              __nv_bfloat16* dst = p.Y + (G.y_row0 + col) * p.ldy + v0;
              if (v0 + 8 <= p.n_vox) {
                __stcs(reinterpret_cast<int4*>(dst), make_int4((int)val.x, (int)val.y, (int)val.z, (int)val.w));
              } else {
                const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&val);
                for (int k = 0; k < 8 && v0 + k < p.n_vox; ++k) dst[k] = v8[k];
              }
            }
          }
          named_bar(1, 32 * kEpiWarps);  // every chunk is read before the tile is written again
        }
      } else {
        // one accumulator per K chunk (one chunk unless the operands are FP32 splits):
        // the first is stored with the bias, later ones are added to the FP32 output
        const int nch = SPLIT ? k_chunks((G.K + kBK - 1) / kBK, chunk_kb) : 1;
        bool alive = true;
        for (int c = 0; c < nch; ++c) {
          if (c > 0) {
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
            const bool okc = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTmemFull);
            if (!__all_sync(0xffffffffu, okc)) {
              alive = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * ACC_STRIDE);
          if (c == 0) {
            // compile-time column loops, so that the bias comes from registers (shuffled)
#pragma unroll
            for (int k0 = 0; k0 < BN / 32; k0 += 4) {
              if (!(32 * k0 + 16 * half < BN && nt * BN + 32 * k0 + 16 * half < G.N)) break;
              uint32_t rv[4][16];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int c0 = 32 * (k0 + u) + 16 * half;
                if (c0 < BN && nt * BN + c0 < G.N) tmem_ld16_nowait(tb + (uint32_t)c0, rv[u]);
              }
              tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int c0 = 32 * (k0 + u) + 16 * half;
                const int nbase = nt * BN + c0;
                if (c0 < BN && nbase < G.N) {
#pragma unroll
                  for (int jj = 0; jj < 16; ++jj) {
                    const int w = 16 * (k0 + u) + jj;
                    const float bv = __shfl_sync(0xffffffffu, breg[(w >> 5) < NBREG ? (w >> 5) : 0], w & 31);
                    const int n = nbase + jj;
                    if (n < G.N && vok) {
                      const int64_t o = (G.y_row0 + n) * p.ldy + vox;
                      const float v = __uint_as_float(rv[u][jj]) + bv;
                      if constexpr (SPLIT)
                        p.Yf[o] = v;
                      else
                        p.Y[o] = __float2bfloat16_rn(v);
                    }
                  }
                }
              }
            }
          } else if constexpr (SPLIT) {
            // later chunks: add to the partial sums this thread stored, their loads all in
            // flight together (no store between them) under the TMEM loads
            for (int k0 = 0; 32 * k0 + 16 * half < BN && nt * BN + 32 * k0 + 16 * half < G.N; ++k0) {
              const int c0 = 32 * k0 + 16 * half, nbase = nt * BN + c0;
              uint32_t rv[16];
              float old[16];
              tmem_ld16_nowait(tb + (uint32_t)c0, rv);
              float* yc = p.Yf + (G.y_row0 + nbase) * p.ldy + vox;
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) old[jj] = (nbase + jj < G.N && vok) ? yc[jj * p.ldy] : 0.f;
              tmem_wait_ld();
#pragma unroll
              for (int jj = 0; jj < 16; ++jj)
                if (nbase + jj < G.N && vok) yc[jj * p.ldy] = old[jj] + __uint_as_float(rv[jj]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            const uint32_t te = CL > 1 ? mapa_shared(tempty_bar(acc), 0) : tempty_bar(acc);
            if (CL > 1)
              mbar_arrive_cluster(te);
            else
              mbar_arrive(te);
          }
        }
        if (!alive) break;
      }
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair frees its TMEM once both epilogues are done with it; after this point no
  // copy, commit or arrival of either CTA targets the other
  if (CL > 1) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if (CL > 1)
      tmem_dealloc_pair(tmem_base, TMEM_COLS);
    else
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
  int n_terms;   // 1 (BF16 operands) or kSplitTerms (three-part splits of FP32 operands)
  int chunk_kb;  // voxel blocks of 64 per accumulation chunk (> 0)
  int64_t tiles_per_split, total_tiles, vps, n_vox, ldp, split_stride;
  int64_t ones_col;  // column of the row sums (rows_in)
  // element (row r, column c) of a split's partial at r * p_rs + c * p_cs: (ldp, 1), or (1, ldp)
  // for the transposed partials of the FP32 path, whose read-modify-write per chunk is then
  // coalesced across a warp's lanes (consecutive rows)
  int64_t p_rs, p_cs;
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

template <int BN, int CL, bool SPLIT>
__host__ __device__ constexpr bool wgrad_sums() { return !SPLIT && CL == 2 && BN / CL + 8 <= 128; }
template <int BN, int CL, bool SPLIT>
__host__ __device__ constexpr int wgrad_b_slot_rows() { return wgrad_sums<BN, CL, SPLIT>() ? BN / CL + 8 : BN / CL; }

// CL = 2: a cluster of two CTAs computes a 256-row x BN tile with 2-SM MMAs:
// each CTA stages its own 128 output rows of dY and BN/2 of the BN input rows
// of X; the even CTA arms the stage barriers and issues the MMAs, each CTA
// drains its own 128 rows.  m_tiles in the groups then counts row-tile pairs.
template <int BN, int STAGES, int CL, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    wgrad_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const __grid_constant__ WgParams p) {
  using namespace ptx;
  static_assert(CL == 1 || CL == 2, "one CTA or a CTA pair");
  static_assert(BN <= 256 && BN % 16 == 0 && (BN / CL) % 8 == 0, "N tile: whole 8-row groups per CTA");
  // SPLIT: FP32 operands as three BF16 planes (3-D maps), six terms, chunked voxels,
  // transposed partials
  const int n_terms = SPLIT ? p.n_terms : 1;
  const int chunk_kb = SPLIT ? p.chunk_kb : (1 << 24);
  // SUMS: the bias-gradient row sums come out of the GEMM itself.  Each CTA's B slot
  // holds 8 constant rows of ones after its BN/CL rows of X; the first column tile of
  // every (split, group, row tile) runs with N = 2 (BN/CL + 8) = 256 instead of BN, and
  // its columns BN/CL .. BN/CL + 7 are sum_v dY[row][v].  (BF16 operands, CTA pairs.)
  constexpr bool SUMS = wgrad_sums<BN, CL, SPLIT>();
  constexpr int B_ROWS = BN / CL;              // rows of X this CTA loads per stage
  constexpr int B_SLOT_ROWS = wgrad_b_slot_rows<BN, CL, SPLIT>();
  constexpr int A_BYTES = 128 * 128;           // 128 rows x 64 voxels
  constexpr int B_BYTES = B_SLOT_ROWS * 128;   // B slot (X rows, then the ones rows)
  constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t TX_BYTES = A_BYTES + B_ROWS * 128;  // bytes the copies deliver per CTA and stage
  constexpr uint32_t TMEM_COLS = 512;          // two accumulators, 256 columns apart
  constexpr uint32_t IDESC = idesc_bf16(128 * CL, BN, false, false);
  constexpr uint32_t IDESC_SUMS = idesc_bf16(128 * CL, 2 * B_SLOT_ROWS, false, false);

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
  const int rank = CL > 1 ? (int)cluster_rank() : 0;
  const int64_t t_first = CL > 1 ? (int64_t)cluster_id_x() : (int64_t)blockIdx.x;
  const int64_t t_step = CL > 1 ? (int64_t)cluster_count_x() : (int64_t)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), CL * kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (SUMS) {
    // the ones rows of every stage (BF16 1.0 pairs), never overwritten by the copies; made
    // visible to the tensor core's proxy before the cluster barrier below
    for (int i = threadIdx.x; i < STAGES * 8 * 32; i += blockDim.x) {
      const int st = i / 256, w = i % 256;
      reinterpret_cast<uint32_t*>(smem + st * STAGE_BYTES + A_BYTES + B_ROWS * 128)[w] = 0x3F803F80u;
    }
    fence_proxy_async_smem();
  }
  if (CL > 1) cluster_sync();  // the peer's barriers exist before any copy or commit reaches them
  if (warp == 1) {
    if (CL > 1) {
      tmem_alloc_pair(smem_u32(tmem_slot), TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
      tmem_relinquish();
    }
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
    for (int64_t t = t_first; t < p.total_tiles && !*abort_flag; t += t_step) {
      int split, g, mt, nt;
      wg_decode(p, t, split, g, mt, nt);
      mt = mt * CL + rank;
      const WgGroup& G = p.g[g];
      const int64_t vs = (int64_t)split * p.vps, ve = min(p.n_vox, vs + p.vps);
      const int nkb = (int)((ve - vs + 63) / 64);
      const int arow = (int)(G.m_row0 + (int64_t)mt * 128);
      const int brow = (int)(G.x_row0 + (int64_t)nt * BN + rank * (BN / CL));
      bool ok = true;
      const int nch = SPLIT ? k_chunks(nkb, chunk_kb) : 1;
      for (int c = 0; c < nch && ok; ++c)
      for (int ti = 0; ti < n_terms && ok; ++ti) {
        const int term = n_terms - 1 - ti;  // smallest part products first
        const int za = split_part_a(term), zb = split_part_b(term);
        for (int kb = c * chunk_kb; kb < min(nkb, (c + 1) * chunk_kb); ++kb) {
          if (!wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, p.err, kErrEmpty)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = sbase + stage * STAGE_BYTES, b_dst = a_dst + A_BYTES;
          const int vx = (int)(vs + (int64_t)kb * 64);
          if (CL > 1) {
            const uint32_t fb = mapa_shared(full_bar(stage), 0);
            if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), CL * TX_BYTES);
            if constexpr (SPLIT) {
              tma_load_3d_pair(&mapA, fb, a_dst, vx, arow, za);
              tma_load_3d_pair(&mapB, fb, b_dst, vx, brow, zb);
            } else {
              tma_load_2d_pair(&mapA, fb, a_dst, vx, arow);
              tma_load_2d_pair(&mapB, fb, b_dst, vx, brow);
            }
          } else {
            mbar_arrive_expect_tx(full_bar(stage), TX_BYTES);
            if constexpr (SPLIT) {
              tma_load_3d(&mapA, full_bar(stage), a_dst, vx, arow, za);
              tma_load_3d(&mapB, full_bar(stage), b_dst, vx, brow, zb);
            } else {
              tma_load_2d(&mapA, full_bar(stage), a_dst, vx, arow);
              tma_load_2d(&mapB, full_bar(stage), b_dst, vx, brow);
            }
          }
          pend[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) break;
    }
    if (rank == 0)
      for (int s = 0; s < STAGES; ++s)
        if (pend[s] >= 0) wait_drain(full_bar(s), (uint32_t)pend[s], p.err, kErrDrain);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int64_t t = t_first; ok && t < p.total_tiles && !*abort_flag; t += t_step) {
      int split, g, mt, nt;
      wg_decode(p, t, split, g, mt, nt);
      const int64_t vs = (int64_t)split * p.vps, ve = min(p.n_vox, vs + p.vps);
      const int nkb = (int)((ve - vs + 63) / 64);
      const int nch = SPLIT ? k_chunks(nkb, chunk_kb) : 1;
      const uint32_t idesc = (SUMS && nt == 0) ? IDESC_SUMS : IDESC;
      for (int c = 0; c < nch; ++c) {
        if (!wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.err, kErrTmemEmpty)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * 256);
        // this chunk's voxel blocks of every term, in the producer's order
        const int nk = SPLIT ? max(0, min(chunk_kb, nkb - c * chunk_kb)) * n_terms : nkb;
        for (int kb = 0; kb < nk; ++kb) {
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
            if (CL > 1)
              mma_bf16_pair(d_tmem, ad, bd, idesc, (kb | k) != 0);
            else
              mma_bf16(d_tmem, ad, bd, idesc, (kb | k) != 0);
          }
          if (CL > 1)
            mma_commit_pair_mc(empty_bar(stage), 0x3);
          else
            mma_commit(empty_bar(stage));
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (CL > 1)
          mma_commit_pair_mc(tfull_bar(acc), 0x3);
        else
          mma_commit(tfull_bar(acc));
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1u;
      }
    }
    if (CL > 1)
      mma_commit_pair(drain_bar);
    else
      mma_commit(drain_bar);
    wait_drain(drain_bar, 0, p.err, kErrDrain);
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;  // 16-column chunks 2k + half
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int64_t t = t_first; t < p.total_tiles; t += t_step) {
      int split, g, mt, nt;
      wg_decode(p, t, split, g, mt, nt);
      mt = mt * CL + rank;
      const WgGroup& G = p.g[g];
      const int m = mt * 128 + q * 32 + lane;
      const int64_t rs = p.p_rs, cs = p.p_cs;
      float* prow = p.P + (int64_t)split * p.split_stride + (G.m_row0 + m) * rs + G.n_col0 * cs;
      const int64_t vs = (int64_t)split * p.vps, ve = min(p.n_vox, vs + p.vps);
      const int nch = SPLIT ? k_chunks((int)((ve - vs + 63) / 64), chunk_kb) : 1;
      bool alive = true;
      // one accumulator per voxel chunk: the first is stored, later ones added (FP32)
      for (int c = 0; c < nch; ++c) {
        bool ok = wait_bounded(tfull_bar(acc), acc_phase, abort_flag, p.err, kErrTmemFull);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          alive = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 256);
        if (SUMS && nt == 0) {
          // N = 256: D column j holds X row j (j < B_ROWS), the row sum (B_ROWS <= j < 128),
          // X row j - 8 (128 <= j < 128 + B_ROWS) or the row sum again
          for (int k0 = 0; 32 * k0 + 16 * half < 2 * B_SLOT_ROWS; k0 += 4) {
            uint32_t rv[4][16];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c0 = 32 * (k0 + u) + 16 * half;
              if (c0 < 2 * B_SLOT_ROWS) tmem_ld16_nowait(tbase + (uint32_t)c0, rv[u]);
            }
            tmem_wait_ld();
            if (m < G.M) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int c0 = 32 * (k0 + u) + 16 * half;
                if (c0 < 2 * B_SLOT_ROWS) {
#pragma unroll
                  for (int j = 0; j < 16; ++j) {
                    const int jc = c0 + j, in_half = jc % B_SLOT_ROWS;
                    const int n = (jc / B_SLOT_ROWS) * B_ROWS + in_half;
                    if (in_half < B_ROWS) {
                      if (n < G.N) prow[n * cs] = __uint_as_float(rv[u][j]);
                    } else if (jc == B_ROWS) {
                      p.P[(int64_t)split * p.split_stride + (G.m_row0 + m) * rs + p.ones_col * cs] =
                          __uint_as_float(rv[u][j]);
                    }
                  }
                }
              }
            }
          }
        } else
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
                if (SPLIT && c > 0) {
                  // later chunks: add to the partial sums this thread stored (loads first)
                  float old[16];
#pragma unroll
                  for (int j = 0; j < 16; ++j) old[j] = nbase + j < G.N ? prow[(nbase + j) * cs] : 0.f;
#pragma unroll
                  for (int j = 0; j < 16; ++j)
                    if (nbase + j < G.N) prow[(nbase + j) * cs] = old[j] + __uint_as_float(rv[u][j]);
                } else {
#pragma unroll
                  for (int j = 0; j < 16; ++j)
                    if (nbase + j < G.N) prow[(nbase + j) * cs] = __uint_as_float(rv[u][j]);
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (CL > 1)
            mbar_arrive_cluster(mapa_shared(tempty_bar(acc), 0));
          else
            mbar_arrive(tempty_bar(acc));
        }
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1u;
      }
      if (!alive) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair frees its TMEM once both epilogues are done with it; after this point no
  // copy, commit or arrival of either CTA targets the other
  if (CL > 1) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if (CL > 1)
      tmem_dealloc_pair(tmem_base, TMEM_COLS);
    else
      tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// host side
// Row sums of dY per voxel split (the bias-gradient column of the weight gradient).
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void __launch_bounds__(256) rowsum_kernel(const T* __restrict__ dY, int64_t lddy, int64_t rows,
                                                     int64_t n_vox, int64_t vps, int splits, float* __restrict__ P,
                                                     int64_t rs, int64_t split_stride, int64_t col_off) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (wid >= rows * splits) return;
  const int64_t row = wid / splits;
  const int split = (int)(wid % splits);
  const int64_t vs = (int64_t)split * vps, ve = min(n_vox, vs + vps);
  const T* r = dY + row * lddy;
  float acc = 0.f;
  // vs is a multiple of 128 and rows are 16-byte aligned: 16-byte vectors up to the last full one
  constexpr int VE = 16 / sizeof(T);
  const int64_t vend = vs + ((ve - vs) / VE) * VE;
  for (int64_t v = vs + (int64_t)lane * VE; v < vend; v += 32 * VE) {
    const uint4 u = *reinterpret_cast<const uint4*>(r + v);
    if constexpr (sizeof(T) == 2) {
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        acc += f.x + f.y;
      }
    } else {
      acc += (__uint_as_float(u.x) + __uint_as_float(u.y)) + (__uint_as_float(u.z) + __uint_as_float(u.w));
    }
  }
  for (int64_t v = vend + lane; v < ve; v += 32) acc += to_f32(r[v]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) P[(int64_t)split * split_stride + row * rs + col_off] = acc;
}

// Three-part BF16 split of an FP32 array (the operands of the FP32 path): part 0 is
// the BF16 rounding of x, part 1 that of the remainder x - x0 (exact in FP32), part
// 2 that of x - x0 - x1.  Each rounding leaves at most 2^-9 of its argument, so
// |x - x0 - x1 - x2| <= 2^-27 |x| (normal range).  Four columns per thread.
__global__ void __launch_bounds__(256) split3_kernel(const float* __restrict__ x, int64_t rows, int64_t cols,
                                                     int64_t ldx, __nv_bfloat16* __restrict__ out, int64_t ldo,
                                                     int64_t part_stride) {
  const int64_t c4 = (ldo + 3) / 4;  // 4-column chunks per output row
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * c4; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / c4, c = (i % c4) * 4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (c + 4 <= cols) {
      const float4 f = *reinterpret_cast<const float4*>(x + r * ldx + c);
      v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
    } else {
      for (int j = 0; j < 4; ++j)
        if (c + j < cols) v[j] = x[r * ldx + c + j];
    }
    __nv_bfloat16 part[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float rem = v[j];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        part[q][j] = __float2bfloat16_rn(rem);
        rem -= __bfloat162float(part[q][j]);
      }
    }
    __nv_bfloat16* o = out + r * ldo + c;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (c + 4 <= ldo) {
        *reinterpret_cast<uint2*>(o + q * part_stride) = *reinterpret_cast<const uint2*>(part[q]);
      } else {
        for (int j = 0; j < 4 && c + j < ldo; ++j) o[q * part_stride + j] = part[q][j];
      }
    }
  }
}

// out[c * ldo + r] = in[r * ldi + c] for r < rows, c < cols (BF16), through 64 x 64 tiles in
// shared memory: the input-gradient GEMM's K-major operator Wt from W.
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int64_t rows,
                                                             int64_t cols, int64_t ldi, __nv_bfloat16* __restrict__ out,
                                                             int64_t ldo) {
  __shared__ __nv_bfloat16 tile[64][66];
  const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int i = ty; i < 64; i += 8) {
    const int64_t r = r0 + i;
#pragma unroll
    for (int j = tx; j < 64; j += 32) {
      const int64_t c = c0 + j;
      tile[i][j] = (r < rows && c < cols) ? in[r * ldi + c] : __float2bfloat16_rn(0.f);
    }
  }
  __syncthreads();
  for (int i = ty; i < 64; i += 8) {
    const int64_t c = c0 + i;
#pragma unroll
    for (int j = tx; j < 64; j += 32) {
      const int64_t r = r0 + j;
      if (c < cols && r < rows) out[c * ldo + r] = tile[j][i];
    }
  }
}

cudaError_t transpose_bf16(const void* in, int64_t rows, int64_t cols, int64_t ldi, void* out, int64_t ldo,
                           cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  TraceScope trace("lsc_transpose_w", st);
  const dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64));
  transpose_bf16_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(in), rows, cols, ldi,
                                              reinterpret_cast<__nv_bfloat16*>(out), ldo);
  count_launch();
  return cudaGetLastError();
}

cudaError_t split_bf16x3(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* out, int64_t ldo,
                         int64_t part_stride, cudaStream_t st) {
  if (rows <= 0 || ldo <= 0) return cudaSuccess;
  TraceScope trace("split_bf16x3", st);
  const int64_t work = rows * ((ldo + 3) / 4);
  const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, 152 * 16);
  split3_kernel<<<blocks, 256, 0, st>>>(x, rows, cols, ldx, reinterpret_cast<__nv_bfloat16*>(out), ldo, part_stride);
  count_launch();
  return cudaGetLastError();
}

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

// BF16 map over a [outer][ld] row-major array using `inner` columns, 128-byte swizzle:
// 2-D, or with part_stride > 0 3-D over the three BF16 parts of a split FP32 operand
// (part_stride elements apart), which the kernels address with the z coordinate.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld_elems, uint32_t box_inner,
              uint32_t box_outer, int64_t part_stride = 0) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint32_t rank = part_stride > 0 ? 3 : 2;
  cuuint64_t dims[3] = {inner, outer, 3};
  cuuint64_t strides[2] = {ld_elems * 2, (uint64_t)part_stride * 2};
  cuuint32_t box[3] = {box_inner, box_outer, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// forward tiles: one staged pass of the full tile (measured faster than two half passes)
constexpr int kFwdPasses = 1;

// operand stages that fit beside the staging tile in the ~226 KiB a CTA may use
template <int BN, bool STAGED, int CL>
constexpr int vox_stages() {
  constexpr int stage = 2 * kBoxBytes + (BN / CL) * 128;
  constexpr int stg = STAGED ? BN / kFwdPasses * 256 : 0;
  constexpr int n = (226 * 1024 - 2048 - stg) / stage;
  return n > 8 ? 8 : n;
}

template <int BN, int STAGES>
constexpr size_t smem_bytes(int a_bytes, int b_bytes) {
  return 1024 + (size_t)STAGES * (a_bytes + b_bytes) + (2 * STAGES + 5) * 8 + 16;
}

// CTAs per cluster of one GEMM: its default unless delimit_set_gemm_cluster forced one
int gemm_cluster(int dflt) {
  const int v = g_gemm_cluster.load();
  return (v == 0 ? dflt : v) == 1 ? 1 : 2;
}

// Clusters of `cl` CTAs of `kern` (with `smem` bytes) that fit on the device at
// once; 0 if the query fails.  Cached per device and kernel.
int max_active_clusters(const void* kern, size_t smem, int cl) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, const void*>, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  for (auto& c : cache)
    if (c.first.first == dev && c.first.second == kern) return c.second;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cl * 64));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache.push_back({{dev, kern}, n});
  return n;
}

// Persistent launch: min(tiles, resident) CTAs (cl = 1) or clusters of cl CTAs.
template <typename... Params, typename... Args>
cudaError_t launch_persistent(void (*kern)(Params...), int64_t tiles, int cl, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cl > 1) {
    const int clusters = max_active_clusters(reinterpret_cast<const void*>(kern), smem, cl);
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3((unsigned)(std::min<int64_t>(tiles, clusters) * cl));
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  } else {
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(tiles, std::max(1, dev_info().sms)));
  }
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  count_launch();
  return e;
}

template <int BN, bool STAGED, int CL, bool SPLIT>
cudaError_t launch_vox(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& my, const VoxParams& p,
                       cudaStream_t st) {
  constexpr int S = vox_stages<BN, STAGED, CL>();
  const size_t smem =
      smem_bytes<BN, S>(2 * kBoxBytes, (BN / CL) * 128) + (STAGED ? BN / kFwdPasses * 256 : 0) + 16;
  auto kern = vox_gemm_kernel<BN, S, STAGED, kFwdPasses, CL, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = launch_persistent(kern, p.total_tiles, CL, smem, st, ma, mb, my, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int BN, bool STAGED, bool SPLIT = false>
cudaError_t launch_vox_cl(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& my, VoxParams& p, int cl,
                          cudaStream_t st) {
  if constexpr ((BN / 2) % 8 == 0) {
    // a pair splits the operator columns: whole 64-column atoms for an MN-major operator
    if (cl > 1 && (p.b_kmajor || (BN / 2) % 64 == 0)) {
      p.total_tiles = (int64_t)((p.m_tiles + 1) / 2) * p.tiles_per_m;
      return launch_vox<BN, STAGED, 2, SPLIT>(ma, mb, my, p, st);
    }
  }
  p.total_tiles = (int64_t)p.m_tiles * p.tiles_per_m;
  return launch_vox<BN, STAGED, 1, SPLIT>(ma, mb, my, p, st);
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
// The operator (B) as stored: MN-major [K rows][N columns] or K-major [N rows][K columns].
struct OperatorView {
  const void* ptr;
  uint64_t rows, cols, ld;  // elements
  bool kmajor;
  int64_t part_stride = 0;  // elements between the BF16 parts of a split FP32 operator (0: BF16)
};

// cl = 2 runs CTA pairs with 2-SM MMAs; a pair splits its bn operator columns
// into two halves of whole 64-column atoms, so bn = 192 becomes 256 there.
cudaError_t run_vox(const CUtensorMap& ma, const OperatorView& B, VoxParams& p, int bn, bool staged_ok, int cl,
                    void* Y, int64_t ldy, cudaStream_t st) {
  if (cl > 1 && bn == 192) bn = 256;
  // MN-major: 64-column x 64-K-row boxes; K-major: 64-K x (bn / cl)-row boxes
  CUtensorMap mb;
  if (!make_map(&mb, B.ptr, B.cols, B.rows, B.ld, 64, B.kmajor ? (uint32_t)(bn / cl) : (uint32_t)kBK, B.part_stride))
    return cudaErrorInvalidValue;
  if (p.n_terms < 1) p.n_terms = 1;
  if (p.chunk_kb < 1) p.chunk_kb = 1 << 24;
  if (p.Yf) staged_ok = false;  // FP32 outputs leave through direct stores
  p.b_kmajor = B.kmajor ? 1 : 0;
  p.tiles_per_m = 0;
  bool same_n = true;
  const int atom = 64 * (cl > 1 && (bn / 2) % 64 == 0 ? 2 : 1);  // last-tile granularity
  for (int i = 0; i < p.n_groups; ++i) {
    p.g[i].n_tiles = (p.g[i].N + bn - 1) / bn;
    const int rem = p.g[i].N - (p.g[i].n_tiles - 1) * bn;
    p.g[i].bn_last = std::min(bn, (rem + atom - 1) / atom * atom);
    p.tiles_per_m += p.g[i].n_tiles;
    same_n = same_n && p.g[i].N == p.g[0].N && p.g[i].y_row0 == (int64_t)i * p.g[0].N;
  }
  p.total_tiles = (int64_t)p.m_tiles * p.tiles_per_m;
  if (p.total_tiles == 0) return cudaSuccess;
  CUtensorMap my;
  memset(&my, 0, sizeof my);
  // the staged copy-out writes 16-byte chunks at voxel offsets that are multiples of 8
  bool staged = staged_ok && same_n && (bn <= 192 || cl > 1) && (reinterpret_cast<uintptr_t>(Y) & 15u) == 0 &&
                ldy % 8 == 0;
  if (staged) {
    switch (bn) {
      case 256: return launch_vox_cl<256, true>(ma, mb, my, p, cl, st);
      case 192: return launch_vox_cl<192, true>(ma, mb, my, p, cl, st);
      default: return launch_vox_cl<128, true>(ma, mb, my, p, cl, st);
    }
  }
  if (p.Yf) {
    switch (bn) {
      case 256: return launch_vox_cl<256, false, true>(ma, mb, my, p, cl, st);
      case 192: return launch_vox_cl<192, false, true>(ma, mb, my, p, cl, st);
      default: return launch_vox_cl<128, false, true>(ma, mb, my, p, cl, st);
    }
  }
  switch (bn) {
    case 256: return launch_vox_cl<256, false>(ma, mb, my, p, cl, st);
    case 240: return launch_vox_cl<240, false>(ma, mb, my, p, cl, st);
    case 192: return launch_vox_cl<192, false>(ma, mb, my, p, cl, st);
    default: return launch_vox_cl<128, false>(ma, mb, my, p, cl, st);
  }
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

bool tc_forward_reads_w(const LscDims& d) { return d.in_blk == (int64_t)d.c_in * d.n_in; }

bool tc_dgrad_reads_wt(const LscDims& d) {
  return d.out_blk == (int64_t)d.c_out * d.n_out && ((int64_t)d.c_in * d.n_in) % kDgradBN == 0;
}

cudaError_t tc_lsc_forward(const LscDims& d, const void* X, const void* W, const void* Wt, const float* bias, void* Y,
                           int64_t n_vox, int64_t ldx, int64_t ldy, int* err, cudaStream_t st, TcParts parts) {
  TraceScope trace(parts.on() ? "lsc_fwd_gemm_f32" : "lsc_fwd_gemm", st);
  CUtensorMap ma;
  if (!make_map(&ma, X, (uint64_t)n_vox, (uint64_t)d.rows_in, (uint64_t)ldx, 64, kBK, parts.act))
    return cudaErrorInvalidValue;
  // Without per-shell column padding the input-feature index of W's columns equals the
  // row index of X, so W serves as the K-major operator and Wt is not needed.
  const bool kmajor = tc_forward_reads_w(d);
  OperatorView B;
  if (kmajor)
    B = OperatorView{W, (uint64_t)d.rows_out, (uint64_t)d.ldW, (uint64_t)d.ldW, true, parts.op};
  else
    B = OperatorView{Wt, (uint64_t)d.rows_in, (uint64_t)d.ldWt, (uint64_t)d.ldWt, false, parts.op};
  VoxParams p;
  memset(&p, 0, sizeof p);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  int Ns[kMaxGroups];
  for (int s = 0; s < d.s_out; ++s) {
    VoxGroup& G = p.g[s];
    G.a_k0 = d.win_lo[s] * per_in;
    G.K = (d.win_hi[s] - d.win_lo[s]) * per_in;
    G.b_n0 = (int)(kmajor ? (int64_t)s * per_out : s * d.out_blk);  // first operator row (K-major) or column
    G.N = per_out;
    G.y_row0 = (int64_t)s * per_out;
    Ns[s] = G.N;
  }
  p.n_groups = d.s_out;
  p.m_tiles = (int)((n_vox + 127) / 128);
  p.n_vox = n_vox;
  p.ldy = ldy;
  p.n_terms = parts.on() ? kSplitTerms : 1;
  p.chunk_kb = parts.on() ? kSplitChunkKb : (1 << 24);
  if (parts.on())
    p.Yf = reinterpret_cast<float*>(Y);
  else
    p.Y = reinterpret_cast<__nv_bfloat16*>(Y);
  p.bias = bias;
  p.err = err;
  // forward tiles are short in K and wide in output: stage the epilogue through TMA stores
  int bn = pick_bn(Ns, d.s_out);
  if (bn == 256) bn = ((Ns[0] % 192) == 0) ? 192 : 128;
  return run_vox(ma, B, p, bn, true, gemm_cluster(2), Y, ldy, st);
}

cudaError_t tc_lsc_dgrad(const LscDims& d, const void* dY, const void* W, const void* Wt, void* dX, int64_t n_vox,
                         int64_t lddy, int64_t lddx, int* err, cudaStream_t st, TcParts parts) {
  TraceScope trace(parts.on() ? "lsc_dgrad_gemm_f32" : "lsc_dgrad_gemm", st);
  CUtensorMap ma;
  if (!make_map(&ma, dY, (uint64_t)n_vox, (uint64_t)d.rows_out, (uint64_t)lddy, 64, kBK, parts.act))
    return cudaErrorInvalidValue;
  // BF16 with Wt available: Wt is the K-major operator (rows = input features, columns = dY
  // rows when W's output blocks carry no padding) and 240-column tiles cover c_in n_in
  // exactly; otherwise W as the MN-major operator (64-column atoms, padded last tile)
  const bool kmajor = !parts.on() && Wt && tc_dgrad_reads_wt(d);
  const OperatorView B = kmajor ? OperatorView{Wt, (uint64_t)d.rows_in, (uint64_t)d.ldWt, (uint64_t)d.ldWt, true}
                                : OperatorView{W, (uint64_t)d.rows_out, (uint64_t)d.ldW, (uint64_t)d.ldW, false,
                                               parts.op};
  VoxParams p;
  memset(&p, 0, sizeof p);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  int Ns[kMaxGroups];
  for (int sp = 0; sp < d.s_in; ++sp) {
    VoxGroup& G = p.g[sp];
    G.a_k0 = d.rwin_lo[sp] * per_out;
    G.K = std::max(0, d.rwin_hi[sp] - d.rwin_lo[sp]) * per_out;
    G.b_n0 = (int)(kmajor ? (int64_t)sp * per_in : sp * d.in_blk);  // first operator row (K-major) or column
    G.N = per_in;
    G.y_row0 = (int64_t)sp * per_in;
    Ns[sp] = G.N;
  }
  p.n_groups = d.s_in;
  p.m_tiles = (int)((n_vox + 127) / 128);
  p.n_vox = n_vox;
  p.ldy = lddx;
  p.n_terms = parts.on() ? kSplitTerms : 1;
  p.chunk_kb = parts.on() ? kSplitChunkKb : (1 << 24);
  if (parts.on())
    p.Yf = reinterpret_cast<float*>(dX);
  else
    p.Y = reinterpret_cast<__nv_bfloat16*>(dX);
  p.bias = nullptr;
  p.err = err;
  const int bn = kmajor ? kDgradBN : pick_bn(Ns, d.s_in);
  return run_vox(ma, B, p, bn, false,
                 gemm_cluster(2), dX, lddx, st);
}

template <int BN, int S, int CL, bool SPLIT>
cudaError_t launch_wgrad(const CUtensorMap& ma, const CUtensorMap& mb, const WgParams& p, cudaStream_t st) {
  const size_t smem = smem_bytes<BN, S>(128 * 128, wgrad_b_slot_rows<BN, CL, SPLIT>() * 128);
  auto kern = wgrad_kernel<BN, S, CL, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = launch_persistent(kern, p.total_tiles, CL, smem, st, ma, mb, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t tc_lsc_wgrad(const LscDims& d, const void* dY, const void* X, float* P, int64_t ldp, int64_t split_stride,
                         int splits, int64_t vps, int64_t n_vox, int64_t lddy, int64_t ldx, int* err, cudaStream_t st,
                         TcParts parts, const void* dY_sum, int64_t lddy_sum) {
  constexpr int BN = kWgradBN;
  const int cl = gemm_cluster(2);
  CUtensorMap ma, mb;
  if (!make_map(&ma, dY, (uint64_t)n_vox, (uint64_t)d.rows_out, (uint64_t)lddy, 64, 128, parts.act))
    return cudaErrorInvalidValue;
  if (!make_map(&mb, X, (uint64_t)n_vox, (uint64_t)d.rows_in, (uint64_t)ldx, 64, BN / cl, parts.act2))
    return cudaErrorInvalidValue;
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
    G.m_tiles = ((G.M + 127) / 128 + cl - 1) / cl;  // tile pairs with clusters of two
    G.n_tiles = (G.N + BN - 1) / BN;
    p.tiles_per_split += (int64_t)G.m_tiles * G.n_tiles;
  }
  p.n_groups = d.s_out;
  p.n_terms = parts.on() ? kSplitTerms : 1;
  p.chunk_kb = parts.on() ? kSplitChunkKb : (1 << 24);
  p.splits = splits;
  p.total_tiles = p.tiles_per_split * splits;
  p.vps = vps;
  p.n_vox = n_vox;
  p.ldp = ldp;
  p.split_stride = split_stride;
  p.p_rs = 1;  // transposed partials: a warp's lanes (consecutive rows) store 128 contiguous bytes
  p.p_cs = ldp;
  p.ones_col = d.rows_in;
  p.P = P;
  p.err = err;
  cudaError_t e = cudaSuccess;
  if (p.total_tiles > 0) {
    TraceScope trace(parts.on() ? "lsc_wgrad_gemm_f32" : "lsc_wgrad_gemm", st);
    // stages: 4 x 46 KiB for one CTA, 7 x 31 KiB per CTA of a pair
    if (parts.on())
      e = cl > 1 ? launch_wgrad<BN, 7, 2, true>(ma, mb, p, st) : launch_wgrad<BN, 4, 1, true>(ma, mb, p, st);
    else
      e = cl > 1 ? launch_wgrad<BN, 7, 2, false>(ma, mb, p, st) : launch_wgrad<BN, 4, 1, false>(ma, mb, p, st);
    if (e != cudaSuccess) return e;
  }
  // bias-gradient column: row sums of dY per split.  BF16 operands on CTA pairs: made by
  // the GEMM (ones rows in its operand slots, one 256-wide column tile per row tile);
  // otherwise a separate HBM-bound pass (a separate N = 16 MMA per step inside the GEMM
  // measured slower: each MMA streams its whole A tile again)
  if (!parts.on() && cl > 1) {
    static_assert(wgrad_sums<BN, 2, false>(), "the BF16 pair kernel makes the row sums");
    return cudaGetLastError();
  }
  const int64_t warps = d.rows_out * splits;
  TraceScope trace_rs("lsc_rowsum", st);
  const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
  if (parts.on())
    rowsum_kernel<float><<<blocks, 256, 0, st>>>(reinterpret_cast<const float*>(dY_sum), lddy_sum, d.rows_out, n_vox,
                                                 vps, splits, P, 1, split_stride, d.rows_in * ldp);
  else
    rowsum_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(dY), lddy, d.rows_out,
                                                         n_vox, vps, splits, P, 1, split_stride, d.rows_in * ldp);
  count_launch();
  return cudaGetLastError();
}

}  // namespace delimit
