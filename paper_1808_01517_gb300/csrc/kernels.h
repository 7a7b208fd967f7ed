// Internal launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

namespace delimit {

constexpr int kMaxGroups = 64;

// One group of a grouped transform: Y[(g,c,i), v] = sum_j T_g[i][j] X[(g,c,j), v]
// with x_row = x_row0 + c * x_cstride + j and y_row = y_row0 + c * y_cstride + i.
struct TransformGroup {
  const float* T;  // n_out x n_in, row-major, FP32
  int64_t x_row0, x_cstride, y_row0, y_cstride;
  int n_in, n_out;
};

struct TransformArgs {
  TransformGroup g[kMaxGroups];
  const void* X;
  void* Y;
  int64_t n_vox, ldx, ldy;
  int channels;
  // gathered input (Signal2SH of masked voxels): output voxel v reads input column
  // index[v] < n_src divided by b0[index[v]] (b0 NULL: no division); err gets a code
  // for an index out of range (that voxel's output is zero)
  const int64_t* index = nullptr;
  const float* b0 = nullptr;
  int64_t n_src = 0;
  int* err = nullptr;
};

// ring-tied weights: expand [n_e][rings+1] -> [n_e][K], or the adjoint (reduce)
cudaError_t launch_ring_weights(const float* src, float* dst, int64_t n_e, int K, int rings, int sectors, bool expand,
                                cudaStream_t st);

// dtype codes as in the C ABI: 0 = F32, 1 = BF16
cudaError_t launch_transform_simt(const TransformArgs& a, int n_groups, int max_out, int in_t, int out_t,
                                  cudaStream_t st);
// the gathered form (a.index set); n_in <= 128 and n_out <= 120 (else cudaErrorInvalidValue)
cudaError_t launch_transform_gather(const TransformArgs& a, int n_groups, int max_out, int in_t, int out_t,
                                    cudaStream_t st);
constexpr int kErrGatherIndex = 0x2100;  // device error word: a gather index outside [0, n_src)
constexpr int kErrWaitProbe = 0x7F00;    // device error word: the bounded-wait self-test ran out

// ---- LSC ----
struct LscDims {
  int s_in, s_out, c_in, c_out, n_in, n_out, K;
  int64_t rows_in, rows_out;  // s_in*c_in*n_in, s_out*c_out*n_out
  // Collapsed operator storage (workspace).  Column blocks are padded to a
  // multiple of 8 elements so that every tile start is 16-byte aligned:
  //   W [rows_out][ldW],  W[(s,co,a)][s'*in_blk + ci*n_in + b]
  //   Wt[rows_in][ldWt], Wt[(s',ci,b)][s*out_blk + co*n_out + a]
  int64_t in_blk, out_blk, ldW, ldWt;
  int64_t m_stride_s, m_stride_sp;  // M of shell pair (s, s'): M + s * m_stride_s + s' * m_stride_sp ([K][N_out][N_in])
  int win_lo[kMaxGroups], win_hi[kMaxGroups];      // input shells [lo, hi) feeding output shell s
  int rwin_lo[kMaxGroups], rwin_hi[kMaxGroups];    // output shells [lo, hi) fed by input shell s'
};

// W[(s,co,a),(s',ci,b)] = sum_k w[co,s,ci,s',k] M_{s,s'}[k][a][b] (0 outside the window and in
// the padding), Wt = W^T (padded layouts above), bias_vec[(s,co,a)] = b[co,s] q[s][a] (0 when b == NULL).
cudaError_t launch_build_w(const LscDims& d, const float* w, const float* b, const float* M, const float* q,
                           void* W, void* Wt, float* bias_vec, int w_t, cudaStream_t st);
// bias_vec alone (the tensor-core operator build writes W itself)
cudaError_t launch_build_bias(const LscDims& d, const float* b, const float* q, float* bias_vec, cudaStream_t st);

// Grouped row-GEMM with the operator stored K-rows x R-columns:
// Y[y_row0 + r, v] = sum_{k<K} At[(at_row0 + k) * ldat + at_col0 + r] X[(x_row0 + k), v] (+ bias[y_row0 + r])
struct RowGemmGroup {
  int64_t at_row0, at_col0, x_row0, y_row0;
  int R, K;
};
struct RowGemmArgs {
  RowGemmGroup g[kMaxGroups];
  const void* At;
  const void* X;
  void* Y;
  const float* bias;  // may be null
  int64_t ldat, ldx, ldy, n_vox;
};
cudaError_t launch_row_gemm_simt(const RowGemmArgs& a, int n_groups, int max_R, int act_t, cudaStream_t st);

// Weight-gradient GEMM: P[split][m_row0 + m][n_col0 + n] = sum_{v in split} dY[m_row0 + m, v] X[x_row0 + n, v]
// for n < N, plus column `ones_col` = sum_v dY[m_row0 + m, v].
struct WgradGroup {
  int64_t m_row0, x_row0, n_col0;
  int M, N;
};
struct WgradArgs {
  WgradGroup g[kMaxGroups];
  const void* dY;
  const void* X;
  float* P;
  int64_t lddy, ldx, ldp, split_stride, n_vox, ones_col;
  int64_t vox_per_split;
};
cudaError_t launch_wgrad_simt(const WgradArgs& a, int n_groups, int max_M, int max_N, int splits, int act_t,
                              cudaStream_t st);

// dw[co,s,ci,s',k] = sum_{a,b} M_{s,s'}[k][a][b] sum_split P[split][(s,co,a)][(s',ci,b)];
// db[co,s] = sum_a q[s][a] sum_split P[split][(s,co,a)][rows_in] (the row sums of dY)
// scratch: reduce_dw_scratch_floats(d) floats of partial sums
size_t reduce_dw_scratch_floats(const LscDims& d);
// P element (row r, column c) of split z at z * split_stride + r * p_rs + c * p_cs; with
// p_rs == 1 (transposed partials of the tensor-core weight gradient) the kernel reads Mt,
// M with a and b swapped per kernel point, so that both streams stay coalesced.
cudaError_t launch_reduce_dw(const LscDims& d, const float* P, int64_t p_rs, int64_t p_cs, int64_t split_stride,
                             int splits, const float* M, const float* Mt, const float* q, float* dw, float* db,
                             float* scratch, cudaStream_t st);

// sets the thread-local message returned by delimit_last_error()
void set_last_error(const std::string& msg);

// Tracing: while enabled (delimit_trace_enable), a TraceScope brackets the launches
// made during its lifetime with CUDA events on `st`, recorded under `name`.
class TraceScope {
 public:
  TraceScope(const char* name, cudaStream_t st);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  int idx_;
  cudaStream_t st_;
};

// host-side count of kernels launched by the library (instrumentation)
void count_launch();
uint64_t launch_count();

}  // namespace delimit
