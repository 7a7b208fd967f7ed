// C ABI of the spherical-layer library (declarations and contracts: include/delimit.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/delimit.h"
#include "host_tables.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace delimit;

namespace {

thread_local std::string g_last_error;

delimit_status fail(delimit_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

delimit_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return DELIMIT_ERR_CUDA;
}

// One device-side error word per device, written by bounded waits.
std::mutex g_err_mu;
int* g_err_word[128] = {nullptr};

int* error_word_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_word[dev]) {
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
    g_err_word[dev] = p;
  }
  return g_err_word[dev];
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tensor-core policy (delimit_set_tensor_cores): 0 CUDA cores only, 1 tensor cores where a
// kernel exists for the call's shape and dtype (else CUDA cores, counted), 2 tensor cores
// required (a call without a tensor-core kernel is refused).
std::atomic<int> g_tc_mode{1};
std::atomic<uint64_t> g_cuda_core_fallbacks{0};

// Called where an activation GEMM is about to run on the CUDA-core kernels.
delimit_status cuda_core_path(const char* what) {
  const int mode = g_tc_mode.load();
  if (mode == 2)
    return fail(DELIMIT_ERR_UNSUPPORTED, std::string(what) +
                                             ": tensor cores are required (delimit_set_tensor_cores(2)) and no "
                                             "tensor-core kernel takes this shape and dtype");
  if (mode == 1) g_cuda_core_fallbacks.fetch_add(1);
  return DELIMIT_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int elem_size(delimit_dtype t) { return t == DELIMIT_BF16 ? 2 : 4; }

bool valid_dtype(delimit_dtype t) { return t == DELIMIT_F32 || t == DELIMIT_BF16; }

// Uploads host float vectors into one device allocation; returns device pointers.
struct Uploader {
  std::vector<float> host;
  std::vector<size_t> offs;
  size_t add(const std::vector<double>& v) {
    size_t o = align_up(host.size(), 64);
    host.resize(o, 0.f);
    for (double x : v) host.push_back(float(x));
    offs.push_back(o);
    return o;
  }
};

}  // namespace

void delimit::set_last_error(const std::string& msg) { g_last_error = msg; }

struct delimit_sh_basis {
  BasisHost h;
  bool on_device = false;
  int device = -1;
  float* d_mem = nullptr;
  struct Dev {
    const float *P, *B, *Pt, *Bt;
  };
  std::vector<Dev> dev;
  int* err_word = nullptr;
  TcBasisTables tc;  // BF16 tensor-core operand images
};

struct delimit_lsc_geometry {
  LscHost h;
  const delimit_sh_basis* ob = nullptr;
  bool on_device = false;
  int device = -1;
  float* d_mem = nullptr;
  const float* d_M = nullptr;  // [S_out][K][N_out][N_in]; resampling-free form [S_out][S_in][K][N_out][N_in]
  const float* d_Mt = nullptr;  // the same with [N_in][N_out] per kernel point (transposed)
  const float* d_q = nullptr;  // [S_out][N_out]
  int* err_word = nullptr;
  LscDims dims_template;  // without channel counts
  FusedTables fused;      // B_s^T of the output basis for the LSC forward with SH2Signal fused
  BuildWTables bw;        // BF16 parts of M for the tensor-core operator build
};

static std::vector<double> transpose(const std::vector<double>& a, int rows, int cols) {
  std::vector<double> t(a.size());
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) t[size_t(c) * rows + r] = a[size_t(r) * cols + c];
  return t;
}

extern "C" {

int delimit_version(void) { return 100; }

uint64_t delimit_kernel_launches(void) { return launch_count(); }

delimit_status delimit_set_tensor_cores(int mode) {
  if (mode < 0 || mode > 2) return fail(DELIMIT_ERR_INVALID_ARG, "tensor-core mode must be 0, 1 or 2");
  g_tc_mode.store(mode);
  tc_set_enabled(mode != 0);
  return DELIMIT_OK;
}

uint64_t delimit_cuda_core_fallbacks(void) { return g_cuda_core_fallbacks.load(); }

delimit_status delimit_set_gemm_cluster(int ctas) {
  if (ctas < 0 || ctas > 2) return fail(DELIMIT_ERR_INVALID_ARG, "GEMM cluster must be 0, 1 or 2");
  tc_set_gemm_cluster(ctas);
  return DELIMIT_OK;
}

const char* delimit_last_error(void) { return g_last_error.c_str(); }

const char* delimit_status_string(delimit_status s) {
  switch (s) {
    case DELIMIT_OK: return "ok";
    case DELIMIT_ERR_INVALID_ARG: return "invalid argument";
    case DELIMIT_ERR_RANK_DEFICIENT: return "rank deficient";
    case DELIMIT_ERR_UNSUPPORTED: return "unsupported";
    case DELIMIT_ERR_ALIGNMENT: return "alignment";
    case DELIMIT_ERR_CUDA: return "cuda error";
    case DELIMIT_ERR_DEVICE_TIMEOUT: return "device timeout";
    case DELIMIT_ERR_OOM: return "out of device memory";
    case DELIMIT_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

delimit_status delimit_sh_basis_create(const double* dirs, const double* bvals, int n_dirs, int order, double lambda,
                                       unsigned flags, delimit_sh_basis** out) {
  if (!out) return fail(DELIMIT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  delimit_sh_basis* b = new (std::nothrow) delimit_sh_basis();
  if (!b) return fail(DELIMIT_ERR_OOM, "host allocation failed");
  std::string err;
  const int rc = build_basis(dirs, bvals, n_dirs, order, lambda, b->h, err, !(flags & DELIMIT_EVAL_ONLY));
  if (rc) {
    delete b;
    return fail(rc == 2 ? DELIMIT_ERR_RANK_DEFICIENT : DELIMIT_ERR_INVALID_ARG, err);
  }
  if (int(b->h.shells.size()) > kMaxGroups) {
    delete b;
    return fail(DELIMIT_ERR_UNSUPPORTED, "more than 64 shells");
  }
  if (!(flags & DELIMIT_HOST_ONLY)) {
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(e, "cudaGetDevice");
    }
    b->err_word = error_word_for_current_device();
    Uploader up;
    const int N = b->h.N;
    std::vector<size_t> o;
    for (auto& s : b->h.shells) {
      o.push_back(up.add(s.P));
      o.push_back(up.add(s.B));
      o.push_back(up.add(transpose(s.P, N, s.m)));
      o.push_back(up.add(transpose(s.B, s.m, N)));
    }
    e = cudaMalloc(&b->d_mem, std::max<size_t>(1, up.host.size()) * sizeof(float));
    if (e != cudaSuccess) {
      delete b;
      return fail(DELIMIT_ERR_OOM, std::string("cudaMalloc tables: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(b->d_mem, up.host.data(), up.host.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(b->d_mem);
      delete b;
      return cuda_fail(e, "cudaMemcpy tables");
    }
    for (size_t s = 0; s < b->h.shells.size(); ++s)
      b->dev.push_back({b->d_mem + o[4 * s], b->d_mem + o[4 * s + 1], b->d_mem + o[4 * s + 2], b->d_mem + o[4 * s + 3]});
    std::string terr;
    if (tc_basis_tables_create(b->h, b->tc, terr) != cudaSuccess) {
      cudaFree(b->d_mem);
      delete b;
      return fail(DELIMIT_ERR_CUDA, "tensor-core tables: " + terr);
    }
    if (tc_basis_tables_create_f32(b->h, b->tc, terr) != cudaSuccess) {
      tc_basis_tables_destroy(b->tc);
      cudaFree(b->d_mem);
      delete b;
      return fail(DELIMIT_ERR_CUDA, "tensor-core FP32 part tables: " + terr);
    }
    b->on_device = true;
  }
  *out = b;
  return DELIMIT_OK;
}

delimit_status delimit_sh_basis_destroy(delimit_sh_basis* b) {
  if (!b) return DELIMIT_OK;
  if (b->on_device) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaFree(b->d_mem);
    tc_basis_tables_destroy_f32(b->tc);
    tc_basis_tables_destroy(b->tc);
    if (cur != b->device && cur >= 0) cudaSetDevice(cur);
  }
  delete b;
  return DELIMIT_OK;
}

delimit_status delimit_sh_basis_info(const delimit_sh_basis* b, int* n_shells, int* n_coef, int* n_dirs) {
  if (!b) return fail(DELIMIT_ERR_INVALID_ARG, "basis is NULL");
  if (n_shells) *n_shells = int(b->h.shells.size());
  if (n_coef) *n_coef = b->h.N;
  if (n_dirs) *n_dirs = b->h.n_dirs;
  return DELIMIT_OK;
}

delimit_status delimit_sh_basis_shell(const delimit_sh_basis* b, int shell, int* n_dirs, int* dir_offset, double* bval) {
  if (!b || shell < 0 || shell >= int(b->h.shells.size())) return fail(DELIMIT_ERR_INVALID_ARG, "bad basis or shell");
  const ShellHost& s = b->h.shells[shell];
  if (n_dirs) *n_dirs = s.m;
  if (dir_offset) *dir_offset = s.dir_off;
  if (bval) *bval = s.bval;
  return DELIMIT_OK;
}

delimit_status delimit_sh_basis_tables(const delimit_sh_basis* b, int shell, double* B, double* P, int* dir_index) {
  if (!b || shell < 0 || shell >= int(b->h.shells.size())) return fail(DELIMIT_ERR_INVALID_ARG, "bad basis or shell");
  const ShellHost& s = b->h.shells[shell];
  if (B) std::memcpy(B, s.B.data(), s.B.size() * sizeof(double));
  if (P) std::memcpy(P, s.P.data(), s.P.size() * sizeof(double));
  if (dir_index) std::memcpy(dir_index, s.dir_index.data(), s.dir_index.size() * sizeof(int));
  return DELIMIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// transforms
// ---------------------------------------------------------------------------
enum TransformKind { kS2SH = 0, kSH2S = 1, kS2SH_BWD = 2, kSH2S_BWD = 3 };

static delimit_status check_device(int device) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != device) return fail(DELIMIT_ERR_INVALID_ARG, "handle was created on another device than the current one");
  return DELIMIT_OK;
}

static delimit_status check_act(const void* p, int64_t ld, int64_t n_vox, delimit_dtype t, const char* name) {
  if (!p) return fail(DELIMIT_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (ld < n_vox) return fail(DELIMIT_ERR_INVALID_ARG, std::string(name) + ": ld < n_vox");
  if (!aligned16(p) || (ld * elem_size(t)) % 16 != 0)
    return fail(DELIMIT_ERR_ALIGNMENT,
                std::string(name) + ": pointer must be 16-byte aligned and ld*sizeof(elem) a multiple of 16");
  return DELIMIT_OK;
}

static delimit_status run_transform(const delimit_sh_basis* b, const void* X, void* Y, int64_t n_vox, int C,
                                    int64_t ldx, int64_t ldy, delimit_dtype in_t, delimit_dtype out_t, void* stream,
                                    TransformKind kind) {
  if (!b) return fail(DELIMIT_ERR_INVALID_ARG, "basis is NULL");
  if (!b->on_device) return fail(DELIMIT_ERR_INVALID_ARG, "basis was created with DELIMIT_HOST_ONLY");
  if (!b->h.has_pinv && (kind == kS2SH || kind == kS2SH_BWD))
    return fail(DELIMIT_ERR_INVALID_ARG, "basis was created with DELIMIT_EVAL_ONLY (no pseudo-inverse)");
  if (n_vox < 0 || C < 1 || C > 65535) return fail(DELIMIT_ERR_INVALID_ARG, "need n_vox >= 0 and 1 <= channels <= 65535");
  if (!valid_dtype(in_t) || !valid_dtype(out_t)) return fail(DELIMIT_ERR_INVALID_ARG, "bad dtype");
  if (n_vox == 0) return DELIMIT_OK;
  delimit_status st = check_device(b->device);
  if (st != DELIMIT_OK) return st;
  if ((st = check_act(X, ldx, n_vox, in_t, "input")) != DELIMIT_OK) return st;
  if ((st = check_act(Y, ldy, n_vox, out_t, "output")) != DELIMIT_OK) return st;
  const int N = b->h.N, S = int(b->h.shells.size());
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  // tensor-core path: BF16 input, N and m_s within the kernel's limits
  if (in_t == DELIMIT_BF16 && tc_transform_supported(b->tc, kind, ldx, ldy, out_t)) {
    cudaError_t e = tc_transform_launch(b->tc, kind, X, Y, n_vox, C, ldx, ldy, out_t, b->err_word, cs);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core transform launch");
    return DELIMIT_OK;
  }
  // FP32 input: three-part BF16 splits made in shared memory, six part products
  if (in_t == DELIMIT_F32 && tc_transform_f32_supported(b->tc, kind, out_t)) {
    cudaError_t e = tc_transform_f32_launch(b->tc, kind, static_cast<const float*>(X), Y, n_vox, C, ldx, ldy, out_t,
                                            b->err_word, cs);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core FP32 transform launch");
    return DELIMIT_OK;
  }
  if ((st = cuda_core_path("transform")) != DELIMIT_OK) return st;
  TransformArgs a{};  // every member zero (or its default)
  int max_out = 0;
  for (int s = 0; s < S; ++s) {
    const ShellHost& sh = b->h.shells[s];
    TransformGroup& g = a.g[s];
    const int64_t sig_row0 = int64_t(C) * sh.dir_off, sig_cs = sh.m;
    const int64_t sh_row0 = int64_t(s) * C * N, sh_cs = N;
    switch (kind) {
      case kS2SH: g.T = b->dev[s].P; g.n_out = N; g.n_in = sh.m;
        g.x_row0 = sig_row0; g.x_cstride = sig_cs; g.y_row0 = sh_row0; g.y_cstride = sh_cs; break;
      case kSH2S: g.T = b->dev[s].B; g.n_out = sh.m; g.n_in = N;
        g.x_row0 = sh_row0; g.x_cstride = sh_cs; g.y_row0 = sig_row0; g.y_cstride = sig_cs; break;
      case kS2SH_BWD: g.T = b->dev[s].Pt; g.n_out = sh.m; g.n_in = N;
        g.x_row0 = sh_row0; g.x_cstride = sh_cs; g.y_row0 = sig_row0; g.y_cstride = sig_cs; break;
      case kSH2S_BWD: g.T = b->dev[s].Bt; g.n_out = N; g.n_in = sh.m;
        g.x_row0 = sig_row0; g.x_cstride = sig_cs; g.y_row0 = sh_row0; g.y_cstride = sh_cs; break;
    }
    max_out = std::max(max_out, g.n_out);
  }
  a.X = X;
  a.Y = Y;
  a.n_vox = n_vox;
  a.ldx = ldx;
  a.ldy = ldy;
  a.channels = C;
  cudaError_t e = launch_transform_simt(a, S, max_out, int(in_t), int(out_t), cs);
  if (e != cudaSuccess) return cuda_fail(e, "transform launch");
  return DELIMIT_OK;
}

extern "C" {

delimit_status delimit_signal2sh(const delimit_sh_basis* b, const void* sig, void* sh, int64_t n_vox, int channels,
                                 int64_t ld_sig, int64_t ld_sh, delimit_dtype in_t, delimit_dtype out_t, void* stream) {
  return run_transform(b, sig, sh, n_vox, channels, ld_sig, ld_sh, in_t, out_t, stream, kS2SH);
}

delimit_status delimit_signal2sh_gather(const delimit_sh_basis* b, const void* dwi, int64_t ld_dwi, int64_t n_src,
                                        const float* b0, const int64_t* index, int64_t n, void* sh, int64_t ld_sh,
                                        int channels, delimit_dtype in_t, delimit_dtype out_t, void* stream) {
  if (!b) return fail(DELIMIT_ERR_INVALID_ARG, "basis is NULL");
  if (!b->on_device) return fail(DELIMIT_ERR_INVALID_ARG, "basis was created with DELIMIT_HOST_ONLY");
  if (!b->h.has_pinv) return fail(DELIMIT_ERR_INVALID_ARG, "basis was created with DELIMIT_EVAL_ONLY (no pseudo-inverse)");
  if (n < 0 || n_src < 1 || channels < 1 || channels > 65535 || ld_dwi < n_src)
    return fail(DELIMIT_ERR_INVALID_ARG, "need n >= 0, n_src >= 1, 1 <= channels <= 65535, ld_dwi >= n_src");
  if (!valid_dtype(in_t) || !valid_dtype(out_t)) return fail(DELIMIT_ERR_INVALID_ARG, "bad dtype");
  if (n == 0) return DELIMIT_OK;
  if (!dwi || !index) return fail(DELIMIT_ERR_INVALID_ARG, "dwi and index must not be NULL");
  delimit_status st = check_device(b->device);
  if (st != DELIMIT_OK) return st;
  if ((st = check_act(sh, ld_sh, n, out_t, "sh")) != DELIMIT_OK) return st;
  const int N = b->h.N, S = int(b->h.shells.size());
  TransformArgs a{};  // every member zero (or its default)
  int max_out = 0;
  for (int s = 0; s < S; ++s) {
    const ShellHost& shl = b->h.shells[s];
    if (shl.m > 128 || N > 120) return fail(DELIMIT_ERR_UNSUPPORTED, "gathered Signal2SH: <= 128 directions per shell, <= 120 coefficients");
    TransformGroup& g = a.g[s];
    g.T = b->dev[s].P;
    g.n_out = N;
    g.n_in = shl.m;
    g.x_row0 = int64_t(channels) * shl.dir_off;
    g.x_cstride = shl.m;
    g.y_row0 = int64_t(s) * channels * N;
    g.y_cstride = N;
    max_out = std::max(max_out, N);
  }
  a.X = dwi;
  a.Y = sh;
  a.n_vox = n;
  a.ldx = ld_dwi;
  a.ldy = ld_sh;
  a.channels = channels;
  a.index = index;
  a.b0 = b0;
  a.n_src = n_src;
  a.err = b->err_word;
  cudaError_t e = launch_transform_gather(a, S, max_out, int(in_t), int(out_t), reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gathered Signal2SH launch");
  return DELIMIT_OK;
}

delimit_status delimit_sh2signal(const delimit_sh_basis* b, const void* sh, void* sig, int64_t n_vox, int channels,
                                 int64_t ld_sh, int64_t ld_sig, delimit_dtype in_t, delimit_dtype out_t, void* stream) {
  return run_transform(b, sh, sig, n_vox, channels, ld_sh, ld_sig, in_t, out_t, stream, kSH2S);
}

delimit_status delimit_signal2sh_backward(const delimit_sh_basis* b, const void* d_sh, void* d_sig, int64_t n_vox,
                                          int channels, int64_t ld_sh, int64_t ld_sig, delimit_dtype in_t,
                                          delimit_dtype out_t, void* stream) {
  return run_transform(b, d_sh, d_sig, n_vox, channels, ld_sh, ld_sig, in_t, out_t, stream, kS2SH_BWD);
}

delimit_status delimit_sh2signal_backward(const delimit_sh_basis* b, const void* d_sig, void* d_sh, int64_t n_vox,
                                          int channels, int64_t ld_sig, int64_t ld_sh, delimit_dtype in_t,
                                          delimit_dtype out_t, void* stream) {
  return run_transform(b, d_sig, d_sh, n_vox, channels, ld_sig, ld_sh, in_t, out_t, stream, kSH2S_BWD);
}

// ---------------------------------------------------------------------------
// LSC
// ---------------------------------------------------------------------------
delimit_status delimit_lsc_geometry_create(const delimit_sh_basis* ob, int order_in, int shells_in, double radius,
                                           int rings, int sectors, int window, unsigned flags,
                                           delimit_lsc_geometry** out) {
  if (!out) return fail(DELIMIT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ob) return fail(DELIMIT_ERR_INVALID_ARG, "out_basis is NULL");
  if (!ob->h.has_pinv) return fail(DELIMIT_ERR_INVALID_ARG, "out_basis was created with DELIMIT_EVAL_ONLY");
  delimit_lsc_geometry* g = new (std::nothrow) delimit_lsc_geometry();
  if (!g) return fail(DELIMIT_ERR_OOM, "host allocation failed");
  std::string err;
  if (flags & ~(DELIMIT_HOST_ONLY | DELIMIT_LSC_NEIGHBOURS)) {
    delete g;
    return fail(DELIMIT_ERR_INVALID_ARG, "unknown geometry flags");
  }
  if (build_lsc(ob->h, order_in, shells_in, radius, rings, sectors, window, (flags & DELIMIT_LSC_NEIGHBOURS) != 0,
                g->h, err)) {
    delete g;
    return fail(DELIMIT_ERR_INVALID_ARG, err);
  }
  if (g->h.s_in > kMaxGroups || g->h.s_out > kMaxGroups) {
    delete g;
    return fail(DELIMIT_ERR_UNSUPPORTED, "more than 64 shells");
  }
  g->ob = ob;
  LscDims& d = g->dims_template;
  std::memset(&d, 0, sizeof d);
  d.s_in = g->h.s_in;
  d.s_out = g->h.s_out;
  d.n_in = g->h.n_in;
  d.n_out = g->h.n_out;
  d.K = g->h.K;
  // collapse matrices of shell pair (s, s') start at s * m_stride_s + s' * m_stride_sp
  const int64_t nkab = int64_t(d.K) * d.n_out * d.n_in;
  d.m_stride_s = g->h.neighbours ? nkab * d.s_in : nkab;
  d.m_stride_sp = g->h.neighbours ? nkab : 0;
  for (int s = 0; s < d.s_out; ++s) {
    int lo = -1, hi = -1;
    for (int p = 0; p < d.s_in; ++p)
      if (g->h.shells[s].window[p]) {
        if (lo < 0) lo = p;
        hi = p + 1;
      }
    d.win_lo[s] = lo;
    d.win_hi[s] = hi;
  }
  for (int p = 0; p < d.s_in; ++p) {
    int lo = -1, hi = -1;
    for (int s = 0; s < d.s_out; ++s)
      if (g->h.shells[s].window[p]) {
        if (lo < 0) lo = s;
        hi = s + 1;
      }
    d.rwin_lo[p] = lo;
    d.rwin_hi[p] = hi;
  }
  if (!(flags & DELIMIT_HOST_ONLY)) {
    if (!ob->on_device) {
      delete g;
      return fail(DELIMIT_ERR_INVALID_ARG, "device geometry needs a device basis");
    }
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess || g->device != ob->device) {
      delete g;
      return fail(DELIMIT_ERR_INVALID_ARG, "geometry must be created on the basis' device");
    }
    g->err_word = error_word_for_current_device();
    // M and q of all output shells, packed densely for the kernels
    std::vector<double> Mall, Mtall, qall;
    for (auto& s : g->h.shells) Mall.insert(Mall.end(), s.M.begin(), s.M.end());
    for (auto& s : g->h.shells) qall.insert(qall.end(), s.q.begin(), s.q.end());
    // Mt: every [N_out][N_in] block of M transposed (the weight-gradient reduction reads it)
    const size_t blk = size_t(d.n_out) * d.n_in;
    Mtall.resize(Mall.size());
    for (size_t o = 0; o < Mall.size(); o += blk)
      for (int a = 0; a < d.n_out; ++a)
        for (int b = 0; b < d.n_in; ++b) Mtall[o + size_t(b) * d.n_out + a] = Mall[o + size_t(a) * d.n_in + b];
    Uploader dense;
    const size_t om = dense.add(Mall), omt = dense.add(Mtall), oqq = dense.add(qall);
    e = cudaMalloc(&g->d_mem, dense.host.size() * sizeof(float));
    if (e != cudaSuccess) {
      delete g;
      return fail(DELIMIT_ERR_OOM, std::string("cudaMalloc geometry: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(g->d_mem, dense.host.data(), dense.host.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(g->d_mem);
      delete g;
      return cuda_fail(e, "cudaMemcpy geometry");
    }
    g->d_M = g->d_mem + om;
    g->d_Mt = g->d_mem + omt;
    g->d_q = g->d_mem + oqq;
    std::string ferr;
    if (fused_tables_create(ob->h, g->fused, ferr) != cudaSuccess) {
      cudaFree(g->d_mem);
      delete g;
      return fail(DELIMIT_ERR_OOM, "fused SH2Signal operator: " + ferr);
    }
    if (build_w_tables_create(g->dims_template, g->d_M, g->bw, ferr) != cudaSuccess) {
      fused_tables_destroy(g->fused);
      cudaFree(g->d_mem);
      delete g;
      return fail(DELIMIT_ERR_OOM, "operator-build tables: " + ferr);
    }
    g->on_device = true;
  }
  *out = g;
  return DELIMIT_OK;
}

delimit_status delimit_lsc_geometry_destroy(delimit_lsc_geometry* g) {
  if (!g) return DELIMIT_OK;
  if (g->on_device) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    cudaFree(g->d_mem);
    fused_tables_destroy(g->fused);
    build_w_tables_destroy(g->bw);
    if (cur != g->device && cur >= 0) cudaSetDevice(cur);
  }
  delete g;
  return DELIMIT_OK;
}

static delimit_status ring_weights(const delimit_lsc_geometry* g, const float* src, float* dst, int c_in, int c_out,
                                   void* stream, bool expand) {
  if (!g) return fail(DELIMIT_ERR_INVALID_ARG, "geometry is NULL");
  if (c_in < 1 || c_out < 1) return fail(DELIMIT_ERR_INVALID_ARG, "need c_in, c_out >= 1");
  if (!src || !dst) return fail(DELIMIT_ERR_INVALID_ARG, "weight pointers must not be NULL");
  if (!g->on_device) return fail(DELIMIT_ERR_INVALID_ARG, "geometry was created with DELIMIT_HOST_ONLY");
  delimit_status st = check_device(g->device);
  if (st != DELIMIT_OK) return st;
  const int64_t n_e = int64_t(c_out) * g->h.s_out * c_in * g->h.s_in;
  cudaError_t e = launch_ring_weights(src, dst, n_e, g->h.K, g->h.rings, g->h.sectors, expand,
                                      reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ring weight launch");
  return DELIMIT_OK;
}

delimit_status delimit_lsc_ring_expand(const delimit_lsc_geometry* g, const float* w_ring, float* w, int c_in, int c_out,
                                       void* stream) {
  return ring_weights(g, w_ring, w, c_in, c_out, stream, true);
}

delimit_status delimit_lsc_ring_reduce(const delimit_lsc_geometry* g, const float* dw, float* dw_ring, int c_in,
                                       int c_out, void* stream) {
  return ring_weights(g, dw, dw_ring, c_in, c_out, stream, false);
}

delimit_status delimit_lsc_geometry_info(const delimit_lsc_geometry* g, int* K, int* n_in, int* n_out, int* s_in,
                                         int* s_out, int64_t* n_nb) {
  if (!g) return fail(DELIMIT_ERR_INVALID_ARG, "geometry is NULL");
  if (K) *K = g->h.K;
  if (n_in) *n_in = g->h.n_in;
  if (n_out) *n_out = g->h.n_out;
  if (s_in) *s_in = g->h.s_in;
  if (s_out) *s_out = g->h.s_out;
  if (n_nb) {
    int64_t t = 0;
    for (auto& s : g->h.shells) t += int64_t(s.nb_indices.size());
    *n_nb = t;
  }
  return DELIMIT_OK;
}

delimit_status delimit_lsc_geometry_tables(const delimit_lsc_geometry* g, int shell, double* kpts, double* M,
                                           double* q, int64_t* nb_indptr, int64_t* nb_indices, int64_t* row_index,
                                           unsigned char* window) {
  if (!g || shell < 0 || shell >= g->h.s_out) return fail(DELIMIT_ERR_INVALID_ARG, "bad geometry or shell");
  const LscShellHost& s = g->h.shells[shell];
  if (kpts) std::memcpy(kpts, s.kpts.data(), s.kpts.size() * sizeof(double));
  if (M) std::memcpy(M, s.M.data(), s.M.size() * sizeof(double));  // [S_in] x K x N_out x N_in when resampling-free
  if (q) std::memcpy(q, s.q.data(), s.q.size() * sizeof(double));
  for (size_t i = 0; nb_indptr && i < s.nb_indptr.size(); ++i) nb_indptr[i] = s.nb_indptr[i];
  for (size_t i = 0; nb_indices && i < s.nb_indices.size(); ++i) nb_indices[i] = s.nb_indices[i];
  if (row_index) {
    const ShellHost& bs = g->ob->h.shells[shell];
    for (int i = 0; i < bs.m; ++i)
      for (int k = 0; k < g->h.K; ++k) row_index[size_t(i) * g->h.K + k] = int64_t(bs.dir_off + i) * g->h.K + k;
  }
  if (window) std::memcpy(window, s.window.data(), s.window.size());
  return DELIMIT_OK;
}

delimit_status delimit_lsc_neighbour_table(const delimit_lsc_geometry* g, int shell, int shell_in, int64_t* indptr,
                                           int64_t* indices, int32_t* bins) {
  if (!g || shell < 0 || shell >= g->h.s_out || shell_in < 0 || shell_in >= g->h.s_in)
    return fail(DELIMIT_ERR_INVALID_ARG, "bad geometry or shell");
  if (!g->h.neighbours) return fail(DELIMIT_ERR_INVALID_ARG, "geometry was not created with DELIMIT_LSC_NEIGHBOURS");
  const LscShellHost& s = g->h.shells[shell];
  const auto& ip = s.pair_indptr[shell_in];
  const auto& ix = s.pair_indices[shell_in];
  const auto& bx = s.pair_bins[shell_in];
  for (size_t i = 0; indptr && i < ip.size(); ++i) indptr[i] = ip[i];
  for (size_t i = 0; indices && i < ix.size(); ++i) indices[i] = ix[i];
  for (size_t i = 0; bins && i < bx.size(); ++i) bins[i] = bx[i];
  return DELIMIT_OK;
}

}  // extern "C"

namespace {

struct LscPlan {
  LscDims d;
  size_t w_bytes;       // one of W / Wt
  size_t off_W, off_Wt, off_bias, off_P, off_dwp, total_fwd, total_bwd;
  // FP32 activations on the tensor cores: three-part BF16 splits of the operator (W3,
  // and Wt3 when the forward reads Wt), of the LSC input (X3) and of dY (dY3); parts of
  // an activation are ld3-strided rows, ld3 = n_vox rounded up to 8
  size_t off_W3, off_Wt3, off_X3, off_dY3;
  int64_t ld3, ldpt;  // ldpt: leading dimension of the transposed weight-gradient partials
  int splits;
  int64_t vox_per_split;
  bool tc;              // tensor-core GEMMs
};

int wgrad_splits(const LscDims& d, int64_t n_vox, int64_t* vps) {
  // The weight-gradient GEMM runs persistent clusters of two CTAs (76 on 152 SMs)
  // over (voxel split, shell, row-tile pair, column tile).  Pick the split count
  // (1..8, each split at least 4096 voxels) whose tile count fills whole waves
  // best; every extra split costs one more FP32 partial of the weight gradient.
  int64_t tiles = 0;
  for (int s = 0; s < d.s_out; ++s) {
    const int64_t M = int64_t(d.c_out) * d.n_out, N = int64_t(d.win_hi[s] - d.win_lo[s]) * d.c_in * d.n_in;
    tiles += ((M + 255) / 256) * ((N + 239) / 240);  // row-tile pairs x 240-column tiles
  }
  tiles = std::max<int64_t>(tiles, 1);
  const int64_t slots = 76;
  const int max_splits = int(std::max<int64_t>(1, std::min<int64_t>(8, n_vox / 4096)));
  int splits = 1;
  double best = 1e30;
  for (int sp = 1; sp <= max_splits; ++sp) {
    const double waves = double((tiles * sp + slots - 1) / slots) / sp;  // in units of one full-K tile
    const double cost = waves * (1.0 + 0.02 * (sp - 1));
    if (cost < best - 1e-9) {
      best = cost;
      splits = sp;
    }
  }
  int64_t per = (n_vox + splits - 1) / splits;
  per = (per + 127) / 128 * 128;
  if (per == 0) per = 128;
  splits = int((n_vox + per - 1) / per);
  if (splits < 1) splits = 1;
  *vps = per;
  return splits;
}

// Whether the operator build writes the transposed operator Wt (the CUDA-core forward
// always reads it; the tensor-core forward only when W's column blocks carry padding).
// The same answer in a forward and the backward that follows keeps
// DELIMIT_LSC_OPERATOR_READY valid between them.  (The BF16 tensor-core input gradient
// transposes W into Wt itself when the build did not write it.)
bool needs_wt(const LscDims& d, bool tc, delimit_dtype t) {
  (void)t;
  return !tc || !tc_forward_reads_w(d);
}

bool make_plan(const delimit_lsc_geometry* g, int64_t n_vox, int c_in, int c_out, delimit_dtype t, LscPlan& p) {
  if (!g || c_in < 1 || c_out < 1 || n_vox < 0 || c_in > 4096 || c_out > 4096 || !valid_dtype(t)) return false;
  p.d = g->dims_template;
  p.d.c_in = c_in;
  p.d.c_out = c_out;
  p.d.rows_in = int64_t(p.d.s_in) * c_in * p.d.n_in;
  p.d.rows_out = int64_t(p.d.s_out) * c_out * p.d.n_out;
  p.d.in_blk = (int64_t(c_in) * p.d.n_in + 7) / 8 * 8;
  p.d.out_blk = (int64_t(c_out) * p.d.n_out + 7) / 8 * 8;
  p.d.ldW = p.d.s_in * p.d.in_blk;
  p.d.ldWt = p.d.s_out * p.d.out_blk;
  const size_t es = elem_size(t);
  const size_t w_bytes = align_up(size_t(p.d.rows_out) * size_t(p.d.ldW) * es, 256);
  const size_t wt_bytes = align_up(size_t(p.d.rows_in) * size_t(p.d.ldWt) * es, 256);
  p.w_bytes = w_bytes;
  p.off_W = 0;
  p.off_Wt = w_bytes;
  p.off_bias = w_bytes + wt_bytes;
  // the operator (W, Wt, bias and, for FP32, their splits) leads both layouts
  const bool f32 = t == DELIMIT_F32;
  p.ld3 = (std::max<int64_t>(n_vox, 1) + 7) / 8 * 8;
  p.off_W3 = p.off_bias + align_up(size_t(p.d.rows_out) * 4, 256);
  p.off_Wt3 = p.off_W3 + (f32 ? align_up(3 * size_t(p.d.rows_out) * size_t(p.d.ldW) * 2, 256) : 0);
  p.off_X3 = p.off_Wt3 +
             (f32 && !tc_forward_reads_w(p.d) ? align_up(3 * size_t(p.d.rows_in) * size_t(p.d.ldWt) * 2, 256) : 0);
  p.total_fwd = p.off_X3 + (f32 ? align_up(3 * size_t(p.d.rows_in) * size_t(p.ld3) * 2, 256) : 0);
  p.splits = wgrad_splits(p.d, std::max<int64_t>(n_vox, 1), &p.vox_per_split);
  p.off_P = p.total_fwd;
  // tensor-core weight gradient: partials written transposed (columns of ldpt floats)
  p.ldpt = (p.d.rows_out + 3) / 4 * 4;
  const size_t p_elems = std::max(size_t(p.d.rows_out) * size_t(p.d.rows_in + 1), size_t(p.d.rows_in + 1) * size_t(p.ldpt));
  p.off_dwp = p.off_P + align_up(size_t(p.splits) * p_elems * 4, 256);
  p.off_dY3 = p.off_dwp + align_up(reduce_dw_scratch_floats(p.d) * 4, 256);
  p.total_bwd = p.off_dY3 + (f32 ? align_up(3 * size_t(p.d.rows_out) * size_t(p.ld3) * 2, 256) : 0);
  p.tc = false;
  return true;
}

// The collapsed operator of one call: W (and Wt where the forward reads it), the bias
// vector when b is given, and for FP32 activations on the tensor cores the BF16
// splits W3 (and Wt3) that the GEMMs read.  The same set whichever call builds it, so
// that DELIMIT_LSC_OPERATOR_READY holds between a forward and its backward.
cudaError_t build_operator(const LscDims& d, const delimit_lsc_geometry* g, const LscPlan& p, const float* w,
                           const float* b, void* W, void* Wt, float* bias, delimit_dtype act_t, bool tc, char* base,
                           cudaStream_t cs) {
  const bool wt = needs_wt(d, tc, act_t);
  if (tc && act_t == DELIMIT_BF16 && !wt && tc_build_w_supported(d, g->bw)) {
    cudaError_t e = tc_build_w(d, g->bw, w, W, g->err_word, cs);
    if (e != cudaSuccess || !bias) return e;
    return launch_build_bias(d, b, g->d_q, bias, cs);
  }
  cudaError_t e = launch_build_w(d, w, b, g->d_M, g->d_q, W, wt ? Wt : nullptr, bias, int(act_t), cs);
  if (e != cudaSuccess || !(tc && act_t == DELIMIT_F32)) return e;
  e = split_bf16x3(static_cast<const float*>(W), d.rows_out, d.ldW, d.ldW, base + p.off_W3, d.ldW, d.rows_out * d.ldW,
                   cs);
  if (e != cudaSuccess || !wt) return e;
  return split_bf16x3(static_cast<const float*>(Wt), d.rows_in, d.ldWt, d.ldWt, base + p.off_Wt3, d.ldWt,
                      d.rows_in * d.ldWt, cs);
}

}  // namespace

extern "C" {

size_t delimit_lsc_workspace_size(const delimit_lsc_geometry* g, int64_t n_vox, int c_in, int c_out,
                                  delimit_dtype act_t, int backward) {
  LscPlan p;
  if (!make_plan(g, n_vox, c_in, c_out, act_t, p)) return 0;
  return backward ? p.total_bwd : p.total_fwd;
}

static delimit_status lsc_common_checks(const delimit_lsc_geometry* g, int64_t n_vox, int c_in, int c_out,
                                        delimit_dtype t, void* ws, size_t ws_bytes, bool bwd, LscPlan& p) {
  if (!g) return fail(DELIMIT_ERR_INVALID_ARG, "geometry is NULL");
  if (!g->on_device) return fail(DELIMIT_ERR_INVALID_ARG, "geometry was created with DELIMIT_HOST_ONLY");
  if (!make_plan(g, n_vox, c_in, c_out, t, p))
    return fail(DELIMIT_ERR_INVALID_ARG, "need n_vox >= 0, 1 <= c_in, c_out <= 4096 and a valid dtype");
  delimit_status st = check_device(g->device);
  if (st != DELIMIT_OK) return st;
  const size_t need = bwd ? p.total_bwd : p.total_fwd;
  if (ws_bytes < need) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "workspace %zu bytes < %zu needed", ws_bytes, need);
    return fail(DELIMIT_ERR_WORKSPACE, buf);
  }
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return fail(DELIMIT_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
  return DELIMIT_OK;
}

delimit_status delimit_lsc_forward(const delimit_lsc_geometry* g, const void* sh_in, const float* w, const float* b,
                                   void* sh_out, int64_t n_vox, int c_in, int c_out, int64_t ld_in, int64_t ld_out,
                                   delimit_dtype act_t, unsigned flags, void* ws, size_t ws_bytes, void* stream) {
  LscPlan p;
  delimit_status st = lsc_common_checks(g, n_vox, c_in, c_out, act_t, ws, ws_bytes, false, p);
  if (st != DELIMIT_OK) return st;
  if (!w) return fail(DELIMIT_ERR_INVALID_ARG, "w is NULL");
  if (n_vox == 0) return DELIMIT_OK;
  if ((st = check_act(sh_in, ld_in, n_vox, act_t, "sh_in")) != DELIMIT_OK) return st;
  if ((st = check_act(sh_out, ld_out, n_vox, act_t, "sh_out")) != DELIMIT_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  void* W = base + p.off_W;
  void* Wt = base + p.off_Wt;
  float* bias = reinterpret_cast<float*>(base + p.off_bias);
  cudaError_t e = cudaSuccess;
  const LscDims& d = p.d;
  const bool tc = tc_gemm_supported(d, n_vox, ld_in, ld_out);
  const bool split = tc && act_t == DELIMIT_F32;  // FP32 on the tensor cores through BF16 splits
  if (!(flags & DELIMIT_LSC_OPERATOR_READY)) {
    e = build_operator(d, g, p, w, b, W, Wt, bias, act_t, tc, base, cs);
    if (e != cudaSuccess) return cuda_fail(e, "LSC operator build launch");
  }
  if (split) {
    void* X3 = base + p.off_X3;
    e = split_bf16x3(static_cast<const float*>(sh_in), d.rows_in, n_vox, ld_in, X3, p.ld3, d.rows_in * p.ld3, cs);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 operand split launch");
    const bool km = tc_forward_reads_w(d);
    TcParts parts;
    parts.act = d.rows_in * p.ld3;
    parts.op = km ? d.rows_out * d.ldW : d.rows_in * d.ldWt;
    e = tc_lsc_forward(d, X3, base + p.off_W3, base + p.off_Wt3, bias, sh_out, n_vox, p.ld3, ld_out, g->err_word, cs,
                       parts);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core FP32 LSC forward launch");
    return DELIMIT_OK;
  }
  if (tc && act_t == DELIMIT_BF16) {
    e = tc_lsc_forward(d, sh_in, W, Wt, bias, sh_out, n_vox, ld_in, ld_out, g->err_word, cs);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core LSC forward launch");
    return DELIMIT_OK;
  }
  if ((st = cuda_core_path("LSC forward")) != DELIMIT_OK) return st;
  RowGemmArgs a;
  std::memset(&a, 0, sizeof a);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  for (int s = 0; s < d.s_out; ++s) {
    RowGemmGroup& gg = a.g[s];
    gg.at_row0 = int64_t(d.win_lo[s]) * per_in;
    gg.at_col0 = int64_t(s) * d.out_blk;
    gg.x_row0 = gg.at_row0;
    gg.y_row0 = int64_t(s) * per_out;
    gg.R = per_out;
    gg.K = (d.win_hi[s] - d.win_lo[s]) * per_in;
  }
  a.At = Wt;
  a.X = sh_in;
  a.Y = sh_out;
  a.bias = bias;
  a.ldat = d.ldWt;
  a.ldx = ld_in;
  a.ldy = ld_out;
  a.n_vox = n_vox;
  e = launch_row_gemm_simt(a, d.s_out, per_out, int(act_t), cs);
  if (e != cudaSuccess) return cuda_fail(e, "LSC forward launch");
  return DELIMIT_OK;
}

delimit_status delimit_lsc_forward_sh2signal_supported(const delimit_lsc_geometry* g, int64_t n_vox, int c_in,
                                                       int c_out, delimit_dtype act_t) {
  LscPlan p;
  if (!g) return fail(DELIMIT_ERR_INVALID_ARG, "geometry is NULL");
  if (!g->on_device) return fail(DELIMIT_ERR_INVALID_ARG, "geometry was created with DELIMIT_HOST_ONLY");
  if (!make_plan(g, n_vox, c_in, c_out, act_t, p))
    return fail(DELIMIT_ERR_INVALID_ARG, "need n_vox >= 0, 1 <= c_in, c_out <= 4096 and a valid dtype");
  if (act_t != DELIMIT_BF16) return fail(DELIMIT_ERR_UNSUPPORTED, "the fused LSC + SH2Signal takes BF16 activations");
  if (const char* why = tc_lsc_fused_unsupported(p.d, g->fused, std::max<int64_t>(n_vox, 1)))
    return fail(DELIMIT_ERR_UNSUPPORTED, std::string("fused LSC + SH2Signal: ") + why);
  return DELIMIT_OK;
}

delimit_status delimit_lsc_forward_sh2signal(const delimit_lsc_geometry* g, const void* sh_in, const float* w,
                                             const float* b, void* sig_out, int64_t n_vox, int c_in, int c_out,
                                             int64_t ld_in, int64_t ld_sig, delimit_dtype act_t, unsigned flags,
                                             void* ws, size_t ws_bytes, void* stream) {
  LscPlan p;
  delimit_status st = lsc_common_checks(g, n_vox, c_in, c_out, act_t, ws, ws_bytes, false, p);
  if (st != DELIMIT_OK) return st;
  if (!w) return fail(DELIMIT_ERR_INVALID_ARG, "w is NULL");
  if (n_vox == 0) return DELIMIT_OK;
  if ((st = delimit_lsc_forward_sh2signal_supported(g, n_vox, c_in, c_out, act_t)) != DELIMIT_OK) return st;
  if ((st = check_act(sh_in, ld_in, n_vox, act_t, "sh_in")) != DELIMIT_OK) return st;
  if ((st = check_act(sig_out, ld_sig, n_vox, act_t, "sig_out")) != DELIMIT_OK) return st;
  const LscDims& d = p.d;
  if (!tc_gemm_supported(d, n_vox, ld_in, ld_sig))
    return fail(DELIMIT_ERR_UNSUPPORTED, "fused LSC + SH2Signal: the tensor-core GEMMs do not take these sizes");
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  void* W = base + p.off_W;
  void* Wt = base + p.off_Wt;
  float* bias = reinterpret_cast<float*>(base + p.off_bias);
  cudaError_t e = cudaSuccess;
  if (!(flags & DELIMIT_LSC_OPERATOR_READY)) {
    e = build_operator(d, g, p, w, b, W, Wt, bias, act_t, true, base, cs);
    if (e != cudaSuccess) return cuda_fail(e, "LSC operator build launch");
  }
  e = tc_lsc_forward_sh2signal(d, g->fused, sh_in, W, bias, sig_out, n_vox, ld_in, ld_sig, g->err_word, cs);
  if (e != cudaSuccess) return cuda_fail(e, "fused LSC + SH2Signal launch");
  return DELIMIT_OK;
}

delimit_status delimit_lsc_backward(const delimit_lsc_geometry* g, const void* sh_in, const float* w, const void* d_out,
                                    void* d_in, float* dw, float* db, int64_t n_vox, int c_in, int c_out, int64_t ld_in,
                                    int64_t ld_out, delimit_dtype act_t, unsigned flags, void* ws, size_t ws_bytes,
                                    void* stream) {
  LscPlan p;
  delimit_status st = lsc_common_checks(g, n_vox, c_in, c_out, act_t, ws, ws_bytes, true, p);
  if (st != DELIMIT_OK) return st;
  const LscDims& d = p.d;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (n_vox == 0) {
    if (dw) {
      cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * size_t(d.c_out) * d.s_out * d.c_in * d.s_in * d.K, cs);
      if (e != cudaSuccess) return cuda_fail(e, "memset dw");
    }
    if (db) {
      cudaError_t e = cudaMemsetAsync(db, 0, sizeof(float) * size_t(d.c_out) * d.s_out, cs);
      if (e != cudaSuccess) return cuda_fail(e, "memset db");
    }
    return DELIMIT_OK;
  }
  if ((st = check_act(d_out, ld_out, n_vox, act_t, "d_out")) != DELIMIT_OK) return st;
  if (dw || db)
    if ((st = check_act(sh_in, ld_in, n_vox, act_t, "sh_in")) != DELIMIT_OK) return st;
  if (d_in) {
    if ((st = check_act(d_in, ld_in, n_vox, act_t, "d_in")) != DELIMIT_OK) return st;
    if (!w) return fail(DELIMIT_ERR_INVALID_ARG, "w is NULL but d_in requested");
  }
  char* base = static_cast<char*>(ws);
  const int per_in = d.c_in * d.n_in, per_out = d.c_out * d.n_out;
  cudaError_t e;
  const bool tc = tc_gemm_supported(d, n_vox, ld_in, ld_out);
  const bool split = tc && act_t == DELIMIT_F32;  // FP32 on the tensor cores through BF16 splits
  void* dY3 = base + p.off_dY3;
  if (split) {
    e = split_bf16x3(static_cast<const float*>(d_out), d.rows_out, n_vox, ld_out, dY3, p.ld3, d.rows_out * p.ld3, cs);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 operand split launch");
  }
  if (d_in) {
    void* W = base + p.off_W;
    void* Wt = base + p.off_Wt;
    if (!(flags & DELIMIT_LSC_OPERATOR_READY)) {
      e = build_operator(d, g, p, w, nullptr, W, Wt, nullptr, act_t, tc, base, cs);
      if (e != cudaSuccess) return cuda_fail(e, "LSC operator build launch");
    }
    bool all_fed = true;
    for (int sp = 0; sp < d.s_in; ++sp) all_fed = all_fed && d.rwin_hi[sp] > d.rwin_lo[sp];
    if (split && all_fed) {
      TcParts parts;
      parts.act = d.rows_out * p.ld3;
      parts.op = d.rows_out * d.ldW;
      e = tc_lsc_dgrad(d, dY3, base + p.off_W3, nullptr, d_in, n_vox, p.ld3, ld_in, g->err_word, cs, parts);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core FP32 LSC input-gradient launch");
    } else if (act_t == DELIMIT_BF16 && all_fed && tc) {
      // the K-major operator of the input gradient: Wt as built, else transposed from W here
      // (a plain transpose: without block padding W is [rows_out][rows_in], Wt [rows_in][rows_out])
      const bool wt_k = tc_dgrad_reads_wt(d);
      if (wt_k && !needs_wt(d, tc, act_t)) {
        e = transpose_bf16(W, d.rows_out, d.ldW, d.ldW, Wt, d.ldWt, cs);
        if (e != cudaSuccess) return cuda_fail(e, "operator transpose launch");
      }
      e = tc_lsc_dgrad(d, d_out, W, wt_k ? Wt : nullptr, d_in, n_vox, ld_out, ld_in, g->err_word, cs);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core LSC input-gradient launch");
    } else {
      if ((st = cuda_core_path("LSC input gradient")) != DELIMIT_OK) return st;
      RowGemmArgs a;
      std::memset(&a, 0, sizeof a);
      for (int sp = 0; sp < d.s_in; ++sp) {
        RowGemmGroup& gg = a.g[sp];
        gg.at_row0 = int64_t(std::max(0, d.rwin_lo[sp])) * per_out;
        gg.at_col0 = int64_t(sp) * d.in_blk;
        gg.x_row0 = gg.at_row0;
        gg.y_row0 = int64_t(sp) * per_in;
        gg.R = per_in;
        gg.K = std::max(0, d.rwin_hi[sp] - d.rwin_lo[sp]) * per_out;
      }
      a.At = W;
      a.X = d_out;
      a.Y = d_in;
      a.bias = nullptr;
      a.ldat = d.ldW;
      a.ldx = ld_out;
      a.ldy = ld_in;
      a.n_vox = n_vox;
      e = launch_row_gemm_simt(a, d.s_in, per_in, int(act_t), cs);
      if (e != cudaSuccess) return cuda_fail(e, "LSC input-gradient launch");
    }
  }
  if (dw || db) {
    float* P = reinterpret_cast<float*>(base + p.off_P);
    const int64_t ldp = d.rows_in + 1;
    int64_t split_stride = d.rows_out * ldp;
    int64_t p_rs = ldp, p_cs = 1;  // row layout (CUDA-core path); the tensor-core path's is transposed
    if (split) {
      void* X3 = base + p.off_X3;
      e = split_bf16x3(static_cast<const float*>(sh_in), d.rows_in, n_vox, ld_in, X3, p.ld3, d.rows_in * p.ld3, cs);
      if (e != cudaSuccess) return cuda_fail(e, "FP32 operand split launch");
      TcParts parts;
      parts.act = d.rows_out * p.ld3;
      parts.act2 = d.rows_in * p.ld3;
      const int64_t ss_t = ldp * p.ldpt;  // transposed partials: rows_in + 1 columns of ldpt floats
      e = tc_lsc_wgrad(d, dY3, X3, P, p.ldpt, ss_t, p.splits, p.vox_per_split, n_vox, p.ld3, p.ld3, g->err_word, cs,
                       parts, d_out, ld_out);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core FP32 LSC weight-gradient launch");
      p_rs = 1;
      p_cs = p.ldpt;
      split_stride = ss_t;
    } else if (act_t == DELIMIT_BF16 && tc) {
      const int64_t ss_t = ldp * p.ldpt;  // transposed partials: rows_in + 1 columns of ldpt floats
      e = tc_lsc_wgrad(d, d_out, sh_in, P, p.ldpt, ss_t, p.splits, p.vox_per_split, n_vox, ld_out, ld_in,
                       g->err_word, cs);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core LSC weight-gradient launch");
      p_rs = 1;
      p_cs = p.ldpt;
      split_stride = ss_t;
    } else {
      if ((st = cuda_core_path("LSC weight gradient")) != DELIMIT_OK) return st;
      WgradArgs a;
      std::memset(&a, 0, sizeof a);
      int maxN = 0;
      for (int s = 0; s < d.s_out; ++s) {
        WgradGroup& gg = a.g[s];
        gg.m_row0 = int64_t(s) * per_out;
        gg.x_row0 = int64_t(d.win_lo[s]) * per_in;
        gg.n_col0 = gg.x_row0;
        gg.M = per_out;
        gg.N = (d.win_hi[s] - d.win_lo[s]) * per_in;
        maxN = std::max(maxN, gg.N);
      }
      a.dY = d_out;
      a.X = sh_in;
      a.P = P;
      a.lddy = ld_out;
      a.ldx = ld_in;
      a.ldp = ldp;
      a.split_stride = split_stride;
      a.n_vox = n_vox;
      a.ones_col = d.rows_in;
      a.vox_per_split = p.vox_per_split;
      e = launch_wgrad_simt(a, d.s_out, per_out, maxN, p.splits, int(act_t), cs);
      if (e != cudaSuccess) return cuda_fail(e, "LSC weight-gradient launch");
    }
    e = launch_reduce_dw(d, P, p_rs, p_cs, split_stride, p.splits, g->d_M, g->d_Mt, g->d_q, dw, db,
                         reinterpret_cast<float*>(base + p.off_dwp), cs);
    if (e != cudaSuccess) return cuda_fail(e, "dw/db reduction launch");
  }
  return DELIMIT_OK;
}

delimit_status delimit_selftest_wait_timeout(void* stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(DELIMIT_ERR_CUDA, "no current CUDA device");
  int* wd = error_word_for_current_device();
  if (!wd) return fail(DELIMIT_ERR_CUDA, "no device error word");
  const cudaError_t e = launch_wait_probe(wd, kErrWaitProbe, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wait probe launch");
  return DELIMIT_OK;
}

delimit_status delimit_device_error(void* stream, int* code) {
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int* wd = error_word_for_current_device();
  if (!wd) return fail(DELIMIT_ERR_CUDA, "no device error word");
  int v = 0;
  e = cudaMemcpy(&v, wd, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read device error word");
  if (code) *code = v;
  if (v) {
    cudaMemset(wd, 0, sizeof(int));
    if (v == kErrGatherIndex) return fail(DELIMIT_ERR_INVALID_ARG, "gathered Signal2SH: an index outside [0, n_src)");
    char buf[96];
    std::snprintf(buf, sizeof buf, "device wait timed out (code 0x%x)", v);
    return fail(DELIMIT_ERR_DEVICE_TIMEOUT, buf);
  }
  return DELIMIT_OK;
}

}  // extern "C"
