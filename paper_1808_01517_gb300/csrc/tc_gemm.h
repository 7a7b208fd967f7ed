// Tensor-core (tcgen05 + TMA, sm_103a) paths of the BF16 layers.
#pragma once

#include <string>

#include "host_tables.h"
#include "kernels.h"

namespace delimit {

// BF16 operand images of one basis' per-shell transform matrices, laid out as
// the tensor-core B operand (K-major, no swizzle), plus launch metadata.
struct TcBasisTables {
  void* d_mem = nullptr;
  int n_shells = 0, N = 0;
  // per shell and per transform kind: byte offset of the image in d_mem, padded sizes
  size_t off[kMaxGroups][4] = {};
  int n_in[kMaxGroups][4] = {}, n_out[kMaxGroups][4] = {}, kpad[kMaxGroups][4] = {}, npad[kMaxGroups][4] = {};
  int m[kMaxGroups] = {}, dir_off[kMaxGroups] = {};
  bool ok = false;
  // FP32 activations: three BF16 parts of every operator (T = T0 + T1 + T2) side by side
  // along the output axis, [kpad][npad3] per shell and kind at byte offset off3 in d_mem3,
  // part q from column q * npad3 / 3 (whole 64-column atoms)
  void* d_mem3 = nullptr;
  size_t off3[kMaxGroups][4] = {};
  int npad3[kMaxGroups][4] = {};
  bool ok3 = false;
};

cudaError_t tc_basis_tables_create(const BasisHost& h, TcBasisTables& t, std::string& err);
void tc_basis_tables_destroy(TcBasisTables& t);
cudaError_t tc_basis_tables_create_f32(const BasisHost& h, TcBasisTables& t, std::string& err);
void tc_basis_tables_destroy_f32(TcBasisTables& t);

// kind: 0 Signal2SH, 1 SH2Signal, 2 Signal2SH adjoint, 3 SH2Signal adjoint (BF16 input)
bool tc_transform_supported(const TcBasisTables& t, int kind, int64_t ldx, int64_t ldy, int out_t);
cudaError_t tc_transform_launch(const TcBasisTables& t, int kind, const void* X, void* Y, int64_t n_vox, int C,
                                int64_t ldx, int64_t ldy, int out_t, int* err_word, cudaStream_t st);
// FP32 input (out_t: 0 = F32, 1 = BF16): each value split into three BF16 parts in shared
// memory, six part products accumulated in FP32 on the tensor cores
bool tc_transform_f32_supported(const TcBasisTables& t, int kind, int out_t);
cudaError_t tc_transform_f32_launch(const TcBasisTables& t, int kind, const float* X, void* Y, int64_t n_vox, int C,
                                    int64_t ldx, int64_t ldy, int out_t, int* err_word, cudaStream_t st);

// LSC GEMMs (BF16 activations, FP32 accumulation in TMEM).
// FP32 activations: every operand is passed as three BF16 parts (split_bf16x3), part p
// at base + p * stride elements (TcParts: stride of the activation operand `act`, of
// the operator `op`), the GEMM accumulates the six leading part products, and the
// outputs of the forward and input-gradient GEMMs are FP32.  TcParts{} = BF16 operands.
struct TcParts {
  int64_t act = 0, op = 0, act2 = 0;  // act2: the weight gradient's second activation (X)
  bool on() const { return act != 0; }
};
bool tc_gemm_supported(const LscDims& d, int64_t n_vox, int64_t ld_in, int64_t ld_out);
// Y[(s,co,a), v] = sum_{k in win(s)} Wt[k][s*out_blk + (co,a)] X[k, v] + bias[(s,co,a)]
// (= sum_k W[(s,co,a)][k] X[k, v]).  When tc_forward_reads_w(d) (no per-shell column
// padding in W) the kernel reads W as a K-major operator and Wt may be absent.
bool tc_forward_reads_w(const LscDims& d);
cudaError_t tc_lsc_forward(const LscDims& d, const void* X, const void* W, const void* Wt, const float* bias, void* Y,
                           int64_t n_vox, int64_t ldx, int64_t ldy, int* err_word, cudaStream_t st,
                           TcParts parts = TcParts{});
// dX[(s',ci,b), v] = sum_{k in rwin(s')} W[k][s'*in_blk + (ci,b)] dY[k, v].  BF16 reads Wt
// (K-major) when tc_dgrad_reads_wt(d) and Wt is given, else W.
bool tc_dgrad_reads_wt(const LscDims& d);
cudaError_t tc_lsc_dgrad(const LscDims& d, const void* dY, const void* W, const void* Wt, void* dX, int64_t n_vox,
                         int64_t lddy, int64_t lddx, int* err_word, cudaStream_t st, TcParts parts = TcParts{});
// P[split][(s,co,a)][(s',ci,b)] = sum_{v in split} dY[(s,co,a), v] X[(s',ci,b), v] for s' in win(s),
// P[split][(s,co,a)][rows_in] = sum_{v in split} dY[(s,co,a), v] (from dY_sum: the BF16 dY, or
// the FP32 dY when the operands are split; lddy_sum its row stride).  The partials are
// stored transposed, P[split][col][row] with leading dimension ldp >= rows_out (the row
// sums in row rows_in), so that the epilogue's stores are coalesced.
cudaError_t tc_lsc_wgrad(const LscDims& d, const void* dY, const void* X, float* P, int64_t ldp, int64_t split_stride,
                         int splits, int64_t vox_per_split, int64_t n_vox, int64_t lddy, int64_t ldx, int* err_word,
                         cudaStream_t st, TcParts parts = TcParts{}, const void* dY_sum = nullptr,
                         int64_t lddy_sum = 0);
// out[c * ldo + r] = in[r * ldi + c] for r < rows, c < cols (BF16)
cudaError_t transpose_bf16(const void* in, int64_t rows, int64_t cols, int64_t ldi, void* out, int64_t ldo,
                           cudaStream_t st);
// out[p * part_stride + r * ldo + c] = part p of x[r * ldx + c] (x = x0 + x1 + x2, each part the
// BF16 rounding of what the earlier parts leave), for r < rows, c < cols; columns [cols, ldo)
// of every part row are zeroed.  ldx a multiple of 4, ldo of 8, both pointers 16-byte aligned.
cudaError_t split_bf16x3(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* out, int64_t ldo,
                         int64_t part_stride, cudaStream_t st);

// The LSC forward with SH2Signal in its epilogue (tc_fused.cu): B_s^T of the output basis'
// shells as the K-major BF16 operator [S][96 directions][64 coefficients], zero-padded.
// Parts of the collapse matrices M_{s,s'} for the tensor-core operator build: three BF16
// parts of every shell pair's [64 kernel points (zero past K)][ldm (a,b) entries] block,
// part q at q * npg * 64 * ldm (ok false: K > 64 or rows too long for the staging tile;
// the CUDA-core build is used).
struct BuildWTables {
  void* d_mp = nullptr;
  int npg = 0, ldm = 0;
  bool ok = false;
};
cudaError_t build_w_tables_create(const LscDims& dims_template, const float* d_M, BuildWTables& t, std::string& err);
void build_w_tables_destroy(BuildWTables& t);
// The BF16 operator W on the tensor cores (zeros outside the window and in the padding);
// supported when K <= 64 and c_in divides 128 (the caller takes it only where the
// forward reads W, i.e. without padding between shell blocks).
bool tc_build_w_supported(const LscDims& d, const BuildWTables& t);
cudaError_t tc_build_w(const LscDims& d, const BuildWTables& t, const float* w, void* W, int* err, cudaStream_t st);

struct FusedTables {
  void* d_b2 = nullptr;
  int shells = 0, m[4] = {}, dir_off[4] = {};
  bool ok = false;  // false: the basis has no fused form (more than 4 shells, 96 directions or 48 coefficients)
};
cudaError_t fused_tables_create(const BasisHost& out_basis, FusedTables& f, std::string& err);
void fused_tables_destroy(FusedTables& f);
// NULL when the fused kernel takes these sizes, else the reason it does not
const char* tc_lsc_fused_unsupported(const LscDims& d, const FusedTables& f, int64_t n_vox);
// S[(s,co,i), v] = sum_a B_s[i][a] bf16(sum_k W[(s,co,a)][k] X[k, v] + bias[(s,co,a)]), BF16 X, W and S;
// W is the K-major collapsed operator (no per-shell padding), S in the signal row layout
cudaError_t tc_lsc_forward_sh2signal(const LscDims& d, const FusedTables& f, const void* X, const void* W,
                                     const float* bias, void* S, int64_t n_vox, int64_t ldx, int64_t lds, int* err,
                                     cudaStream_t st);

// one CTA waiting on an mbarrier nothing arrives at, through the kernels' bounded wait:
// after the limit (2 s) the error word gets `code` and the kernel returns
cudaError_t launch_wait_probe(int* err, int code, cudaStream_t st);

// process-wide switch (default on): when off every BF16 step runs on the CUDA-core kernels
void tc_set_enabled(bool on);
bool tc_enabled();
void tc_set_gemm_cluster(int cl);  // 0 = each GEMM's default, 1 or 2 CTAs per cluster

}  // namespace delimit
