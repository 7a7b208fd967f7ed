/*
 * delimit.h - C ABI of the GB300 (sm_103a) DELIMIT spherical-layer library.
 *
 * Koppers & Merhof, "DELIMIT PyTorch - An extension for Deep Learning in
 * Diffusion Imaging" (arXiv:1808.01517).  The library implements the paper's
 * three layers: Signal2SH and SH2Signal (Sec. 2.2) and the local spherical
 * convolution, LSC (Sec. 2.3, including "Extension to multiple b-values").
 *
 * Conventions shared by every call
 * --------------------------------
 * Activations follow the paper's 5-D tensor convention (Sec. 2.1:
 * subjects x (#shells * #directions) x H x W x D): a tensor is a row-major
 * matrix whose ROWS are features and whose COLUMNS are voxels, voxels
 * contiguous.  `n_vox` columns are used; consecutive rows are `ld` elements
 * apart (ld >= n_vox).  Row order:
 *   signal rows  (s, c, i): row = C * dir_off[s] + c * m_s + i
 *                (shell s, channel c, direction i of shell s)
 *   SH rows      (s, c, j): row = (s * C + c) * N + j
 *                (N = (L+1)(L+2)/2 coefficients, j = l(l+1)/2 + m)
 * With C = 1 this is exactly the paper's tensor for one subject.
 * Alignment: every activation pointer must be 16-byte aligned and
 * ld * sizeof(element) a multiple of 16 (DELIMIT_ERR_ALIGNMENT otherwise).
 *
 * Ownership: handles own their host FP64 tables and device copies and are
 * immutable after creation.  Activation, weight and workspace pointers are
 * caller-owned device memory; no compute call allocates.  Calls are
 * asynchronous on `stream` (a cudaStream_t passed as void*; NULL is the legacy
 * default stream).  Argument errors are returned synchronously; errors of a
 * running kernel (a bounded device-side wait that ran out) are reported by
 * delimit_device_error().  All entry points are thread-safe for distinct
 * handles; delimit_last_error() is per thread.
 * Per-device state: the library resolves some device addresses once per device
 * and keeps them for the life of the process (the device error word, and the
 * scratch array of delimit_lsc_forward_noalloc).  Neither they nor any handle
 * survive cudaDeviceReset() or the destruction of the device's primary context:
 * do not use the library on a device after resetting it.
 *
 * Shells: rows of a gradient table are grouped by b-value rounded to an
 * integer, shells in ascending b, rows of a shell in input order
 * (delimit_sh_basis_tables returns the original row of every grouped row).
 * b <= 0 rows are rejected: the paper normalises by the b = 0 volume first
 * (Sec. 2.2) and the caller does that.
 */
#ifndef DELIMIT_H
#define DELIMIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DELIMIT_OK = 0,
  DELIMIT_ERR_INVALID_ARG = 1,     /* bad size, order, direction, null pointer, ... */
  DELIMIT_ERR_RANK_DEFICIENT = 2,  /* normal equations singular (e.g. lambda = 0, m < N) */
  DELIMIT_ERR_UNSUPPORTED = 3,     /* valid request outside what this library implements */
  DELIMIT_ERR_ALIGNMENT = 4,       /* pointer or row stride violates the 16-byte rule */
  DELIMIT_ERR_CUDA = 5,            /* a CUDA runtime call failed (see delimit_last_error) */
  DELIMIT_ERR_DEVICE_TIMEOUT = 6,  /* a bounded device-side wait ran out */
  DELIMIT_ERR_OOM = 7,             /* device table allocation failed at create time */
  DELIMIT_ERR_WORKSPACE = 8        /* workspace smaller than *_workspace_size() */
} delimit_status;

typedef enum {
  DELIMIT_F32 = 0,  /* float32 activations, FP32 arithmetic (the accurate path) */
  DELIMIT_BF16 = 1  /* bfloat16 activations, tensor cores, FP32 accumulation */
} delimit_dtype;

/* create flags */
#define DELIMIT_HOST_ONLY 1u /* build host FP64 tables only (no device copies, no GPU needed) */
#define DELIMIT_EVAL_ONLY 2u /* basis for SH2Signal only: no pseudo-inverse (P reads as zero); any
                                direction count and lambda = 0 allowed.  Signal2SH, its adjoint and
                                LSC geometries reject such a basis with INVALID_ARG.  SH2Signal in
                                Sec. 2.2 takes only sh_order and gradients. */

/* LSC shell windows (which input shells s' feed output shell s) */
/* Geometry flag: the LSC without resampling (the alternative that Sec. 2.3 argues
 * against), see delimit_lsc_geometry_create. */
#define DELIMIT_LSC_NEIGHBOURS 4u

#define DELIMIT_WINDOW_SAME 0      /* s' = s (needs as many input as output shells) */
#define DELIMIT_WINDOW_ADJACENT 1  /* |s - s'| <= 1 (same) */
#define DELIMIT_WINDOW_ALL (-1)    /* every input shell: the paper's shells-as-channels form */

typedef struct delimit_sh_basis delimit_sh_basis;
typedef struct delimit_lsc_geometry delimit_lsc_geometry;

/* ------------------------------------------------------------------------ */
/* Spherical-harmonic basis of one gradient table (Sec. 2.2, Signal2SH      */
/* parameters sh_order, gradients, lb_lambda).                               */
/* ------------------------------------------------------------------------ */

/* Builds, per shell s, the real even-order SH basis B_s[i, j] = Y_j(g_i)
 * (Descoteaux 2007, cited in Sec. 1) and the Laplace-Beltrami regularised
 * pseudo-inverse P_s = (B_s^T B_s + lambda diag(l^2 (l+1)^2))^-1 B_s^T in FP64
 * (Cholesky), then uploads FP32/BF16 copies unless DELIMIT_HOST_ONLY.
 *   dirs   host, n_dirs x 3 doubles, each of norm 1 +- 1e-6
 *   bvals  host, n_dirs doubles, every one > 0
 *   order  even, 0..16;  lambda >= 0
 * Errors: INVALID_ARG (odd/negative order, bad norm, b <= 0, lambda < 0,
 * null pointer), RANK_DEFICIENT (a shell's normal matrix is not positive
 * definite), OOM / CUDA on device upload.  *out is NULL on error. */
delimit_status delimit_sh_basis_create(const double* dirs, const double* bvals, int n_dirs, int order,
                                       double lambda, unsigned flags, delimit_sh_basis** out);
delimit_status delimit_sh_basis_destroy(delimit_sh_basis* basis);

/* Sizes: number of shells, coefficients N, total directions. Any out pointer may be NULL. */
delimit_status delimit_sh_basis_info(const delimit_sh_basis* basis, int* n_shells, int* n_coef,
                                     int* n_dirs);

/* One shell: directions m_s, offset dir_off[s] of its first grouped row, its b-value. */
delimit_status delimit_sh_basis_shell(const delimit_sh_basis* basis, int shell, int* n_dirs,
                                      int* dir_offset, double* bval);

/* Host FP64 copies of shell s: B (m_s x N, row-major), P (N x m_s, row-major) and
 * dir_index (m_s ints: original row of each grouped row).  NULL skips an output. */
delimit_status delimit_sh_basis_tables(const delimit_sh_basis* basis, int shell, double* B, double* P,
                                       int* dir_index);

/* Signal2SH (Sec. 2.2): sh[(s,c,:), v] = P_s sig[(s,c,:), v] for every shell s,
 * channel c < channels and voxel v < n_vox.  in_t/out_t: F32 or BF16 each.
 * sig: signal rows, sh: SH rows (layout above).  n_vox = 0 does nothing.
 * Arithmetic (all four transforms): tcgen05 tensor cores with FP32 accumulation.
 * BF16 input is multiplied as stored by the BF16 operator; F32 input is split in
 * shared memory into three BF16 parts (x = x0 + x1 + x2 to 2^-27 |x|), the
 * operator likewise on the host, and the six part products down to 2^-18 of the
 * leading one are accumulated (FP32-level error).  Shapes beyond the tensor-core
 * kernels (more than 256 directions or coefficients in a shell, more than 8
 * shells) run on CUDA cores under the policy of delimit_set_tensor_cores.
 * Errors: INVALID_ARG (NULL basis or pointer, n_vox < 0, channels outside
 * 1..65535, ld < n_vox, a host-only or evaluation-only basis, a basis made on
 * another device), ALIGNMENT (16-byte rule), CUDA (launch failure). */
delimit_status delimit_signal2sh(const delimit_sh_basis* basis, const void* sig, void* sh, int64_t n_vox,
                                 int channels, int64_t ld_sig, int64_t ld_sh, delimit_dtype in_t,
                                 delimit_dtype out_t, void* stream);

/* SH2Signal (Sec. 2.2): sig[(s,c,:), v] = B_s sh[(s,c,:), v] on the basis' own
 * directions (create a basis on the "resampled" directions to evaluate there).
 * Errors as delimit_signal2sh, an evaluation-only basis being allowed here. */
delimit_status delimit_sh2signal(const delimit_sh_basis* basis, const void* sh, void* sig, int64_t n_vox,
                                 int channels, int64_t ld_sh, int64_t ld_sig, delimit_dtype in_t,
                                 delimit_dtype out_t, void* stream);

/* Signal2SH of selected voxels of a volume with the b = 0 normalisation fused into
 * the load (Sec. 2.2: the signal is divided by the b = 0 image before fitting):
 *   sh[(s,c,:), k] = P_s dwi[(s,c,:), index[k]] / b0[index[k]]   for k < n.
 *   dwi    device, signal rows (channels x directions, layout above) x n_src
 *          voxels, row stride ld_dwi elements, dtype in_t (no alignment rule)
 *   b0     device float32 [n_src] (voxels with b0 <= 0 give zero coefficients),
 *          or NULL for an already normalised signal
 *   index  device int64 [n], source voxels (e.g. from delimit_mask_compact); an
 *          index outside [0, n_src) gives zero coefficients and sets the device
 *          error word (delimit_device_error, code 0x2100)
 *   sh     device, SH rows x n, ld_sh (16-byte rule), dtype out_t
 * Errors: INVALID_ARG (null pointers, sizes), UNSUPPORTED (more than 128
 * directions in a shell or more than 120 coefficients). */
delimit_status delimit_signal2sh_gather(const delimit_sh_basis* basis, const void* dwi, int64_t ld_dwi,
                                        int64_t n_src, const float* b0, const int64_t* index, int64_t n,
                                        void* sh, int64_t ld_sh, int channels, delimit_dtype in_t,
                                        delimit_dtype out_t, void* stream);

/* Adjoints used by back-propagation: d_sig = P_s^T d_sh and d_sh = B_s^T d_sig, same
 * layouts, dtypes and errors as the forward calls (the Signal2SH adjoint needs the
 * pseudo-inverse, so it refuses an evaluation-only basis). */
delimit_status delimit_signal2sh_backward(const delimit_sh_basis* basis, const void* d_sh, void* d_sig,
                                          int64_t n_vox, int channels, int64_t ld_sh, int64_t ld_sig,
                                          delimit_dtype in_t, delimit_dtype out_t, void* stream);
delimit_status delimit_sh2signal_backward(const delimit_sh_basis* basis, const void* d_sig, void* d_sh,
                                          int64_t n_vox, int channels, int64_t ld_sig, int64_t ld_sh,
                                          delimit_dtype in_t, delimit_dtype out_t, void* stream);

/* ------------------------------------------------------------------------ */
/* Local spherical convolution (Sec. 2.3; multi-shell form of Sec. 2.3.1).   */
/* ------------------------------------------------------------------------ */

/* Geometry of one LSC layer.  Output shell s is sampled on out_basis' shell-s
 * directions ("sampled_gradients"); its output order and lambda ("sh_order_out",
 * "lb_lambda") are out_basis'.  The input is SH of order `order_in` on
 * `shells_in` shells.  Kernel: origin plus `rings` rings of `sectors` points,
 * ring r = 1..rings at polar angle r * radius / rings ("angular_distance",
 * "kernel_sizes"), K = 1 + rings * sectors points in the order
 * [origin, ring 1 (azimuth 0, 2pi/sectors, ...), ring 2, ...], tangent frame
 * e1 = normalise(a - (a.g) g) with a the axis of smallest |g_k| (lowest k on
 * ties), e2 = g x e1.  Built in FP64: kernel points, the input basis at every
 * kernel point, M_{s,k} = P_out,s B^K_{s,k} (N_out x N_in), q_s = P_out,s 1,
 * the window table and the neighbour table {j : |g_i.g_j| >= cos(radius)}.
 *
 * flags: DELIMIT_HOST_ONLY (host tables only), DELIMIT_LSC_NEIGHBOURS (the
 * resampling-free form): input shell s' is sampled on out_basis' shell-s'
 * directions (shells_in must equal its shell count); each acquired neighbour j
 * of output direction i in shell s' (|g_i.g_j| >= cos(radius)), oriented onto
 * g_i's hemisphere, is binned to the kernel point of i nearest to it (largest
 * dot product, lowest k on ties); a kernel point takes the mean of its
 * neighbours' values (0 when it has none) and meets the kernel weights as in the
 * resampled form.  The collapse is then per shell pair,
 * M_{s,s',k} = P_out,s A^{s,s'}_k B_in,s' (A_k the bin means), and the forward,
 * backward and workspace calls are unchanged.
 * Errors: INVALID_ARG (radius outside (0, pi/2], rings/sectors < 1, window not
 * matching the shell counts, bad order, unknown flags, resampling-free tables
 * over 256 MiB), OOM/CUDA on upload. */
delimit_status delimit_lsc_geometry_create(const delimit_sh_basis* out_basis, int order_in, int shells_in,
                                           double radius, int rings, int sectors, int window,
                                           unsigned flags, delimit_lsc_geometry** out);
delimit_status delimit_lsc_geometry_destroy(delimit_lsc_geometry* geom);

/* Sizes: kernel points K, coefficients in/out, shells in/out, neighbour-table
 * entries summed over output shells.  Any out pointer may be NULL. */
delimit_status delimit_lsc_geometry_info(const delimit_lsc_geometry* geom, int* K, int* n_coef_in,
                                         int* n_coef_out, int* shells_in, int* shells_out,
                                         int64_t* n_neighbours);

/* Host copies of output shell s's tables; NULL skips an output.
 *   kpts       m_s x K x 3 doubles (kernel points)
 *   M          K x N_out x N_in doubles (M_{s,k}); resampling-free geometries:
 *              shells_in x K x N_out x N_in (M_{s,s',k})
 *   q          N_out doubles
 *   nb_indptr  m_s + 1 int64, nb_indices nb_indptr[m_s] int64 (ascending)
 *   row_index  m_s x K int64: row (dir_off[s] + i) * K + k of kernel point (i, k)
 *   window     shells_in bytes: 1 where input shell s' feeds output shell s */
delimit_status delimit_lsc_geometry_tables(const delimit_lsc_geometry* geom, int shell, double* kpts,
                                           double* M, double* q, int64_t* nb_indptr, int64_t* nb_indices,
                                           int64_t* row_index, unsigned char* window);

/* Resampling-free geometries only: the acquired neighbours of every direction of
 * output shell `shell` among the directions of input shell `shell_in` (host
 * arrays; NULL skips one): indptr m_s + 1 int64, indices indptr[m_s] int64
 * (ascending within a direction), bins indptr[m_s] int32, the kernel point
 * 0..K-1 each neighbour is binned to.  INVALID_ARG for another geometry or a
 * shell out of range. */
delimit_status delimit_lsc_neighbour_table(const delimit_lsc_geometry* geom, int shell, int shell_in,
                                           int64_t* indptr, int64_t* indices, int32_t* bins);

/* Ring-tied (isotropic) kernels: one weight for the origin and one per ring,
 * shared by the ring's points, the circularly symmetric form of the cyclic
 * kernel (Sec. 2.3):
 *   w[co,s,ci,s',k] = w_ring[co,s,ci,s',ring(k)],  ring(0) = 0,
 *   ring(k) = 1 + (k - 1) / sectors for k >= 1 (kernel point order: origin, ring 1, ...).
 * delimit_lsc_ring_expand writes the per-point weights w [c_out, S_out, c_in,
 * S_in, K] that delimit_lsc_forward / _backward take from w_ring [c_out, S_out,
 * c_in, S_in, rings + 1]; delimit_lsc_ring_reduce is its adjoint (dw_ring[r] =
 * sum of dw over ring r's points, fixed order), turning the weight gradient of
 * delimit_lsc_backward into the ring weights' gradient.  Device float32 arrays;
 * asynchronous on `stream`.  With more sectors than the input SH order the layer
 * then acts on each SH band l of every channel pair as the multiplier
 * w0 + sectors * sum_r w_r P_l(cos(r alpha / rings)) followed by the output
 * projection, independent of the tangent frames. */
delimit_status delimit_lsc_ring_expand(const delimit_lsc_geometry* geom, const float* w_ring, float* w, int c_in,
                                       int c_out, void* stream);
delimit_status delimit_lsc_ring_reduce(const delimit_lsc_geometry* geom, const float* dw, float* dw_ring, int c_in,
                                       int c_out, void* stream);

/* LSC call flags.  DELIMIT_LSC_OPERATOR_READY: `workspace` already holds the
 * collapsed operator (and, for a forward, the bias vector) built by an earlier
 * forward or backward call with the same geometry, sizes, dtype, w and b; the
 * call skips rebuilding it.  The operator sits at the start of the workspace in
 * both layouts, so a backward may reuse the workspace of the forward it
 * follows (give the forward a backward-sized workspace). */
#define DELIMIT_LSC_OPERATOR_READY 1u

/* Device workspace bytes needed by delimit_lsc_forward (backward = 0) or
 * delimit_lsc_backward (backward = 1) for these sizes; 0 on invalid input. */
size_t delimit_lsc_workspace_size(const delimit_lsc_geometry* geom, int64_t n_vox, int c_in, int c_out,
                                  delimit_dtype act_t, int backward);

/* LSC forward (Sec. 2.3): for every voxel, resample each input shell's SH
 * interpolant at the kernel points of every output-shell direction, take the
 * point-wise product with the kernel weights summed over kernel points, input
 * channels and windowed input shells, add the bias, and project onto SH of
 * the output order.  Computed through the exact linear collapse
 * sh_out[(s,co,:)] = sum_{ci, s' in win(s)} (sum_k w[co,s,ci,s',k] M_{s,k}) sh_in[(s',ci,:)]
 *                    + b[co,s] q_s.
 *   sh_in   device, SH rows (S_in x c_in x N_in) x n_vox, ld_in
 *   w       device float32 [c_out, S_out, c_in, S_in, K] (entries outside the window unused)
 *   b       device float32 [c_out, S_out], or NULL for no bias
 *   sh_out  device, SH rows (S_out x c_out x N_out) x n_vox, ld_out
 *   act_t   dtype of sh_in and sh_out
 *   flags   0 or DELIMIT_LSC_OPERATOR_READY (the workspace already holds this
 *           call's collapsed operator and bias vector; see above)
 *   workspace >= delimit_lsc_workspace_size(..., 0) bytes, 256-byte aligned.
 * BF16 runs on tcgen05 (FP32 accumulation).  F32 runs on tcgen05 too: the
 * input, the operator and (backward) the upstream gradient are split into
 * three BF16 parts each (x = x0 + x1 + x2 to 2^-27 |x|), the six part products
 * down to 2^-18 of the leading one are accumulated in FP32, and K is summed in
 * chunks of 1,024 whose results are added in FP32 (measured error against
 * FP64 about 1e-6 at 65,536 voxels, 16 -> 64 channels); with
 * delimit_set_tensor_cores(0) F32 runs as FP32 FMA on CUDA cores.  The F32
 * workspace includes the split copies (3 x 2 bytes per element of sh_in, the
 * operator and, backward, d_out).
 * Errors: INVALID_ARG (NULL geometry or w, a host-only geometry or one made on
 * another device, n_vox < 0, c_in or c_out outside 1..4096, ld < n_vox),
 * WORKSPACE (ws_bytes below the size above; checked before anything else runs,
 * also for n_vox = 0, which then does nothing), ALIGNMENT (workspace not 256-byte
 * aligned, or an activation breaking the 16-byte rule), CUDA (launch failure). */
delimit_status delimit_lsc_forward(const delimit_lsc_geometry* geom, const void* sh_in, const float* w,
                                   const float* b, void* sh_out, int64_t n_vox, int c_in, int c_out,
                                   int64_t ld_in, int64_t ld_out, delimit_dtype act_t, unsigned flags,
                                   void* workspace, size_t ws_bytes, void* stream);

/* The LSC forward followed by SH2Signal on the output basis' directions, in one kernel
 * (Sec. 2.3: the paper's LSC example pipes SH -> LSC -> SH2Signal; Sec. 2.2 for
 * SH2Signal):
 *   sig_out[(s,co,i), v] = sum_a B_s[i][a] c_out[(s,co,a), v],   c_out as delimit_lsc_forward,
 * with B_s the SH basis of output shell s at its own directions (the geometry's output
 * basis) and c_out rounded to BF16 where the unfused pair stores it.  c_out is never
 * written to memory.
 *   sig_out  device, signal rows (s, co, i) of the output basis (S_out shells, c_out
 *            channels, m_s directions each) x n_vox, row stride ld_sig (16-byte rule)
 *   other arguments as delimit_lsc_forward (workspace: delimit_lsc_workspace_size(..., 0);
 *   DELIMIT_LSC_OPERATOR_READY likewise)
 * Runs on the tcgen05 tensor cores only: BF16 activations, c_out a multiple of 4, at most
 * 48 output coefficients (order 8), 96 directions per output shell and 4 output shells,
 * c_in * N_in a multiple of 8.  Other requests return DELIMIT_ERR_UNSUPPORTED with the
 * reason (check first with delimit_lsc_forward_sh2signal_supported) and callers run
 * delimit_lsc_forward + delimit_sh2signal instead.  Errors otherwise as
 * delimit_lsc_forward. */
delimit_status delimit_lsc_forward_sh2signal(const delimit_lsc_geometry* geom, const void* sh_in, const float* w,
                                             const float* b, void* sig_out, int64_t n_vox, int c_in, int c_out,
                                             int64_t ld_in, int64_t ld_sig, delimit_dtype act_t, unsigned flags,
                                             void* workspace, size_t ws_bytes, void* stream);
/* OK when delimit_lsc_forward_sh2signal takes these sizes on this device, UNSUPPORTED
 * (reason in delimit_last_error) when not, INVALID_ARG for invalid sizes. */
delimit_status delimit_lsc_forward_sh2signal_supported(const delimit_lsc_geometry* geom, int64_t n_vox, int c_in,
                                                       int c_out, delimit_dtype act_t);

/* LSC backward for upstream gradient d_out (SH rows of the output):
 *   d_in  = adjoint of the forward in sh_in (same layout as sh_in), or NULL
 *   dw    = float32 [c_out, S_out, c_in, S_in, K] (zero outside the window), or NULL
 *   db    = float32 [c_out, S_out], or NULL
 *   flags = DELIMIT_LSC_OPERATOR_READY reuses the operator a forward with the same
 *   geometry, sizes, dtype and w built in this workspace (b is not needed here).
 * All outputs are overwritten (not accumulated).  Reductions over voxels are
 * deterministic (fixed split and order).
 *   workspace >= delimit_lsc_workspace_size(..., 1) bytes, 256-byte aligned.
 * n_vox = 0 writes zeros to dw and db.  w is needed only for d_in, sh_in only for
 * dw or db.  Errors as delimit_lsc_forward, with d_out, sh_in and d_in checked
 * like its activations. */
delimit_status delimit_lsc_backward(const delimit_lsc_geometry* geom, const void* sh_in, const float* w,
                                    const void* d_out, void* d_in, float* dw, float* db, int64_t n_vox,
                                    int c_in, int c_out, int64_t ld_in, int64_t ld_out, delimit_dtype act_t,
                                    unsigned flags, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Helpers of the learned network and whole-volume inference (no counterpart */
/* in the paper beyond its use of the layers inside networks, Sec. 2 and 3)  */
/* ------------------------------------------------------------------------ */

/* y = x > 0 ? x : slope * x on `rows` feature rows of `n_vox` voxels (activation
 * between LSC layers, applied to SH coefficients).  x and y may alias. */
delimit_status delimit_leaky_relu(const void* x, void* y, int64_t rows, int64_t n_vox, int64_t ld_x, int64_t ld_y,
                                  float slope, delimit_dtype dtype, void* stream);
/* dx = dy * (y > 0 ? 1 : slope), with y the forward output (it keeps the input's sign). */
delimit_status delimit_leaky_relu_backward(const void* y, const void* dy, void* dx, int64_t rows, int64_t n_vox,
                                           int64_t ld_y, int64_t ld_dy, int64_t ld_dx, float slope,
                                           delimit_dtype dtype, void* stream);

/* Table T5: index[0..*count) = ascending positions i < n with mask[i] != 0 (the
 * brain-mask voxel list of a volume stored with its last axis fastest).  Device
 * pointers; *count is written on the device.  index must hold n entries in the
 * worst case.  Deterministic.  workspace >= delimit_mask_compact_workspace_size(n). */
size_t delimit_mask_compact_workspace_size(int64_t n);
delimit_status delimit_mask_compact(const uint8_t* mask, int64_t n, int64_t* index, int64_t* count, void* workspace,
                                    size_t ws_bytes, void* stream);

/* dst[r, j] = src[r, index[j]] for r < rows, j < n (volume -> masked voxel list);
 * indices outside [0, n_src) give 0.  scatter is the inverse placement
 * dst[r, index[j]] = src[r, j] (indices outside [0, n_dst) are skipped). */
delimit_status delimit_gather_voxels(const void* src, int64_t ld_src, int64_t n_src, int64_t rows, const int64_t* index,
                                     int64_t n, void* dst, int64_t ld_dst, delimit_dtype dtype, void* stream);
delimit_status delimit_scatter_voxels(const void* src, int64_t ld_src, int64_t rows, const int64_t* index, int64_t n,
                                      void* dst, int64_t ld_dst, int64_t n_dst, delimit_dtype dtype, void* stream);

/* Same computation as delimit_lsc_forward, for callers that cannot allocate
 * device memory where they run the layer (inside a region where the CUDA
 * allocator must not be called, such as a host callback or a stream another
 * component is capturing; hosts whose allocator owns all device memory; or
 * deployments with a fixed memory budget), so they cannot supply a workspace.
 * The paper has no counterpart to this call.
 * Scratch: a fixed 16 MiB (16777216-byte) device array inside this library,
 * present on every GPU that loads the library until the process exits.  Sizes
 * whose forward workspace (delimit_lsc_workspace_size(..., 0)) exceeds it are
 * rejected with DELIMIT_ERR_WORKSPACE and a message; nothing is allocated,
 * neither here nor in the kernels it launches.  The first call on a device
 * (with that device current) resolves the array's device address; make that
 * first call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents (every call rewrites what it reads): calls
 * that overlap on the GPU (different streams, or host threads without
 * ordering) race on it and must be serialised by the caller. */
delimit_status delimit_lsc_forward_noalloc(const delimit_lsc_geometry* geom, const void* sh_in, const float* w,
                                           const float* b, void* sh_out, int64_t n_vox, int c_in, int c_out,
                                           int64_t ld_in, int64_t ld_out, delimit_dtype act_t, void* stream);

/* ------------------------------------------------------------------------ */
/* Errors and version                                                        */
/* ------------------------------------------------------------------------ */

/* Synchronises `stream`, then reads and clears the device error word that
 * bounded device-side waits set when they run out (and a gathered Signal2SH sets
 * for an index out of range, code 0x2100).  *code receives the raw word (0 =
 * none).  Returns DEVICE_TIMEOUT for a wait that ran out, INVALID_ARG for code
 * 0x2100, CUDA if the synchronisation failed, OK otherwise. */
delimit_status delimit_device_error(void* stream, int* code);

/* Self-test of the bounded device waits (no counterpart in the paper): launches one
 * CTA on `stream` whose thread waits, through the same bounded wait the tensor-core
 * kernels use, on an mbarrier that nothing arrives at.  After the wait limit (2 s) it
 * records code 0x7F00 in the device error word and returns, so that the next
 * delimit_device_error reports DEVICE_TIMEOUT and the context stays usable.  Returns
 * CUDA if the launch fails. */
delimit_status delimit_selftest_wait_timeout(void* stream);

/* Process-wide tensor-core policy for the activation GEMMs (the transforms and
 * the three LSC GEMMs); no counterpart in the paper.
 *   1 (default): each call runs on the tcgen05 tensor-core kernels when one
 *     takes its shape and dtype (BF16 directly, F32 as BF16 part splits), else
 *     on the CUDA-core kernels; every such call is counted by
 *     delimit_cuda_core_fallbacks().
 *   2: tensor cores required: a call that would run on the CUDA cores returns
 *     DELIMIT_ERR_UNSUPPORTED (with the step named in delimit_last_error())
 *     before launching anything.
 *   0: every step on the CUDA-core kernels (same results within the dtype's
 *     rounding; used to cross-check the two).
 * Other values: INVALID_ARG.  The operator build runs on the tensor cores for
 * BF16 activations when K <= 64, c_in divides 128 and c_in * N_in is a multiple
 * of 8 (modes 1 and 2), else on the CUDA cores; it, the weight-gradient reduction and the gathered Signal2SH
 * are not counted as fallbacks and never refused. */
delimit_status delimit_set_tensor_cores(int mode);

/* Process-wide CTA-pair choice of the LSC tensor-core GEMMs (forward, input and
 * weight gradients); no counterpart in the paper.
 *   0 (default): each GEMM's own choice: CTA pairs issuing 2-SM MMAs where the
 *     operator tiles split into two whole halves, else single CTAs.
 *   2: CTA pairs wherever the tiles allow (as 0 for the shapes above);
 *   1: single-CTA MMAs everywhere (the form the other shapes take; results equal
 *     to the pairs' up to FP32 summation order).
 * Other values: INVALID_ARG.  Takes effect at the next call. */
delimit_status delimit_set_gemm_cluster(int ctas);

/* Number of activation-GEMM calls that ran on the CUDA cores under policy 1
 * since the process started (host-side count).  No counterpart in the paper. */
uint64_t delimit_cuda_core_fallbacks(void);

/* Tracing: while enabled, every group of kernel launches made by a call is
 * bracketed by CUDA events recorded on the call's stream.  Enabling (or
 * disabling) clears the record.  delimit_trace_summary synchronises on the
 * recorded events and writes JSON {"name": {"n": launches, "ms": total device
 * time}, ...} into buf (truncated to cap - 1 characters); it returns the full
 * length.  Names: signal2sh_tc, sh2signal_tc, signal2sh_bwd_tc,
 * sh2signal_bwd_tc (the _f32 suffix for FP32 input), transform_simt, lsc_build_w
 * (lsc_build_w_tc on the tensor cores), lsc_fwd_gemm, lsc_dgrad_gemm,
 * lsc_wgrad_gemm (the _f32 suffix for split FP32 operands), lsc_fwd_sh2signal (the
 * fused LSC forward + SH2Signal), lsc_rowsum (FP32 and
 * single-CTA paths), split_bf16x3, lsc_reduce_dw, lsc_gemm_simt, lsc_wgrad_simt.
 * No counterpart in the paper. */
delimit_status delimit_trace_enable(int enable);
int64_t delimit_trace_summary(char* buf, size_t cap);

/* Number of CUDA kernels this library has launched in the process so far
 * (host-side count, for instrumentation).  No counterpart in the paper. */
uint64_t delimit_kernel_launches(void);

const char* delimit_status_string(delimit_status status);
const char* delimit_last_error(void); /* detail of the last failure on this thread */
int delimit_version(void);            /* major * 10000 + minor * 100 + patch */

#ifdef __cplusplus
}
#endif

#endif /* DELIMIT_H */
