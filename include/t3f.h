/*
 * t3f.h -- C ABI of the GB300 (sm_103a) Tensor-Train sweep library.
 *
 * The library computes the batched, core-by-core transfer-matrix sweeps of the T3F method
 * (Novikov et al., "Tensor Train decomposition on TensorFlow", JMLR 2020) on one GPU:
 * inner products / Gram matrices / norms, element gather with the completion loss,
 * TT-matrix x TT-vector, Householder orthogonalisation and the Riemannian tangent-space
 * projection project_sum, each with a hand-written adjoint.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - TT format (paper, Section 1): core k of a TT-vector has shape (r_{k-1}, n_k, r_k),
 *    of a TT-matrix (r_{k-1}, m_k, n_k, r_k), with r_0 = r_d = 1; indices are 0-based.
 *  - Batch layout ("packed"): a t3f_tt describes `batch` objects of identical shape whose
 *    cores live in ONE device buffer. Core k of all objects forms a contiguous block of
 *    batch * r_{k-1} * m_k * n_k * r_k elements (m_k = 1 for TT-vectors), row-major in
 *    [batch][r_{k-1}][m_k][n_k][r_k]; the blocks follow each other for k = 0..d-1 with no
 *    padding. t3f_packed_size() gives the element count.
 *  - Ownership: the caller owns every device buffer (inputs, outputs, workspace). The
 *    library allocates nothing and keeps no state between calls. Host arrays inside a
 *    descriptor (n, m, ranks) are read during the call only.
 *  - Streams: all device work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *    default stream). Calls are asynchronous; a returned status reports argument checks
 *    and launch errors only. Outputs are overwritten, never accumulated.
 *  - Workspace: t3f_workspace_size() returns the bytes an operation needs for the given
 *    descriptors; a smaller `ws_bytes` returns T3F_ERR_WORKSPACE before any launch. The
 *    workspace must be 256-byte aligned.
 *  - Errors: every entry point validates its descriptors (NULL pointers, d range, rank
 *    boundary conditions, shape agreement, dtype) and returns a negative t3f_status without
 *    launching anything when a check fails. t3f_status_string() names a status.
 *  - Precision: storage dtype is per descriptor. The sweeps accumulate in FP32; the QR of
 *    t3f_orthogonalize and the final norm / loss reductions run in FP64.
 */
#ifndef T3F_H
#define T3F_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* t3f_stream_t; /* identical to cudaStream_t */

typedef enum {
  T3F_OK = 0,
  T3F_ERR_ARG = -1,         /* NULL pointer, negative size, d out of range, bad enum */
  T3F_ERR_SHAPE = -2,       /* ranks/modes/batches of the operands disagree */
  T3F_ERR_DTYPE = -3,       /* storage type not supported by this entry point */
  T3F_ERR_WORKSPACE = -4,   /* ws_bytes below t3f_workspace_size() or misaligned ws */
  T3F_ERR_CUDA = -5,        /* a CUDA launch or runtime call failed */
  T3F_ERR_TIMEOUT = -6,     /* a bounded device-side wait ran out (see t3f_device_status) */
  T3F_ERR_UNSUPPORTED = -7  /* valid request beyond this build's kernel limits (e.g. rank) */
} t3f_status;

typedef enum { T3F_F32 = 0, T3F_F64 = 1, T3F_BF16 = 2 } t3f_dtype;

/* Arithmetic of the bulk sweeps: FP32 CUDA cores, or tensor cores with FP32 accumulation. */
typedef enum { T3F_MATH_FP32 = 0, T3F_MATH_TF32 = 1, T3F_MATH_BF16 = 2 } t3f_math;

#define T3F_MAX_D 64      /* maximum number of cores */
#define T3F_MAX_RANK 64   /* maximum TT-rank handled by the sweep kernels */
#define T3F_MAX_MODE 4096 /* maximum mode size n_k (and m_k) */

/* A batch of TT-vectors (m == NULL) or TT-matrices (m != NULL) of one shape. */
typedef struct {
  int32_t batch;          /* number of objects, >= 1 */
  int32_t d;              /* number of cores, 1 <= d <= T3F_MAX_D */
  const int32_t* m;       /* host [d] row modes of a TT-matrix, or NULL for a TT-vector */
  const int32_t* n;       /* host [d] (column) modes, each in [1, T3F_MAX_MODE] */
  const int32_t* ranks;   /* host [d+1] TT-ranks, ranks[0] = ranks[d] = 1 */
  void* cores;            /* device pointer to the packed cores (layout above) */
  int32_t dtype;          /* t3f_dtype of the cores */
} t3f_tt;

/* Operation ids for t3f_workspace_size(). */
typedef enum {
  T3F_OP_GRAM = 1, T3F_OP_GRAM_BWD = 2, T3F_OP_NORM = 3,
  T3F_OP_GATHER = 4, T3F_OP_GATHER_BWD = 5, T3F_OP_RGATHER_BWD = 6,
  T3F_OP_MATVEC = 7, T3F_OP_MATVEC_BWD = 8,
  T3F_OP_ORTH = 9, T3F_OP_PSUM = 10, T3F_OP_PSUM_BWD = 11,
  T3F_OP_PROJECT = 12, T3F_OP_TANGENT_GRAM = 13, T3F_OP_COMPLETION_HVP = 14,
  T3F_OP_ROUND = 15, T3F_OP_GRAM_BWD_TC = 16
} t3f_op;

/* Name of a status code (static string). */
const char* t3f_status_string(int32_t status);

/* Library version, major*10000 + minor*100 + patch. */
int32_t t3f_version(void);

/* Number of CUDA kernels this library has launched in the process so far (every launch
 * site counts one, successful or not); used to report kernel launch counts. */
int64_t t3f_launch_count(void);

/* Number of elements of the packed cores of `t` (0 if the descriptor is invalid). */
int64_t t3f_packed_size(const t3f_tt* t);

/*
 * Workspace bytes for operation `op`:
 *   GRAM, GRAM_BWD: a = A, b = B.          NORM: a = A, b unused.
 *   GATHER, GATHER_BWD: a = X, n_items = N tuples.
 *   RGATHER_BWD: a = U (left-orthogonal form), b = V, n_items = N.
 *   MATVEC, MATVEC_BWD: a = A (TT-matrix), b = x.
 *   ORTH: a = X.    PSUM, PSUM_BWD, PROJECT: a = U, b = Z (the batch being projected).
 *   TANGENT_GRAM: a = dA, b = dB.   COMPLETION_HVP: a = U, b = V, n_items = N.
 *   ROUND: a = X.    GRAM_BWD_TC: a = A, b = B (t3f_gram_backward with math TF32 or BF16).
 * Returns 0 for an invalid request (check with the call itself for the status).
 */
size_t t3f_workspace_size(int32_t op, const t3f_tt* a, const t3f_tt* b, int64_t n_items);

/*
 * Gram matrix (paper Section 4, 'gram'; batch broadcasting of Section 3.1):
 * G[a * B->batch + b] = <A_a, B_b> = sum over all elements of full(A_a) * full(B_b),
 * computed by the left transfer sweep M_0 = 1, M_k = sum_i A_k[:,i,:]^T M_{k-1} B_k[:,i,:].
 * A, B: TT-vectors with equal d and n_k (else T3F_ERR_SHAPE); F32 or BF16 cores; ranks may
 * differ between A and B. G: device float [A->batch][B->batch]. math: t3f_math --
 *   FP32: CUDA-core FP32 arithmetic throughout.
 *   TF32 (F32 cores) / BF16 (F32 or BF16 cores): the two products of every sweep step run on
 *   the tensor cores with operands rounded to TF32 / BF16 (round to nearest) and FP32
 *   accumulation; ranks <= 64 (zero-padded to 16, 32 or 64), else T3F_ERR_UNSUPPORTED.
 * ws: t3f_workspace_size(T3F_OP_GRAM) bytes (the error word; may be NULL for FP32). A
 * tensor-core wait that runs out writes T3F_ERR_TIMEOUT there (see t3f_device_status).
 */
t3f_status t3f_gram(const t3f_tt* A, const t3f_tt* B, float* G, int32_t math,
                    void* ws, size_t ws_bytes, t3f_stream_t stream);

/*
 * Frobenius norms (paper Section 4, 'norm'): out[a] = sqrt(<A_a, A_a>) in FP64.
 * out: device double [A->batch].
 */
t3f_status t3f_norm(const t3f_tt* A, double* out, void* ws, size_t ws_bytes,
                    t3f_stream_t stream);

/*
 * Adjoint of t3f_gram: given dG (device float [A->batch][B->batch]), writes the cotangents
 * of sum_ab dG[a,b] <A_a, B_b>:
 *   dA_a^k[:,i,:] = sum_b dG[a,b] M^{ab}_{k-1} B_b^k[:,i,:] (R^{ab}_{k+1})^T,
 *   dB_b^k[:,i,:] = sum_a dG[a,b] (M^{ab}_{k-1})^T A_a^k[:,i,:] R^{ab}_{k+1},
 * with R the right transfer sweep. The partials are recomputed inside (nothing is kept from
 * the forward call). dA, dB: F32 descriptors with the shapes of A and B. Either may be NULL
 * to skip it. math (t3f_math):
 *   FP32: CUDA-core FP32 throughout; ws: t3f_workspace_size(T3F_OP_GRAM_BWD) bytes.
 *   TF32 (F32 cores) / BF16 (F32 or BF16 cores): tensor cores (tcgen05, FP32 accumulation)
 *   in tiles of (128/RA) x (128/RB) pairs, ranks <= 64 (zero-padded to 16, 32 or 64), else
 *   T3F_ERR_UNSUPPORTED. The left and right sweeps store the partials of every interface
 *   (M scaled by dG) in the workspace, rounded to the operand type; then per (tile, core,
 *   side) the products T = gM Y_i and dX_i = T R^T run on the tensor cores. ws:
 *   t3f_workspace_size(T3F_OP_GRAM_BWD_TC) bytes (error word first; a tensor-core wait that
 *   runs out writes T3F_ERR_TIMEOUT there, see t3f_device_status).
 */
t3f_status t3f_gram_backward(const t3f_tt* A, const t3f_tt* B, const float* dG,
                             t3f_tt* dA, t3f_tt* dB, int32_t math, void* ws, size_t ws_bytes,
                             t3f_stream_t stream);

/*
 * Element gather (paper Section 1, completion example): for N index tuples
 * idx (device int32, layout [d][N]), vals[t] = X(idx[0][t], ..., idx[d-1][t]) for the
 * single TT X (X->batch must be 1, F32 cores). Indices out of [0, n_k) give T3F_ERR_ARG
 * only if detected on the host; on the device they are clamped into range and counted in
 * the workspace error word (t3f_device_status).
 * y: device float [N] or NULL. vals: device float [N] or NULL. loss: device double [1] or
 * NULL; when given, loss = 1/2 sum_t (vals_t - y_t)^2 (y required).
 */
t3f_status t3f_gather(const t3f_tt* X, const int32_t* idx, int64_t N, const float* y,
                      float* vals, double* loss, void* ws, size_t ws_bytes,
                      t3f_stream_t stream);

/*
 * Allocation-free t3f_gather (no counterpart in the paper; an interface convenience).
 * Same arguments and results as t3f_gather without the workspace: for callers that cannot
 * allocate device memory -- e.g. a plugin whose host framework owns all device memory
 * through its own pool or a hard cap, or code that must avoid the implicit device
 * synchronisation of cudaMalloc/cudaFree. The scratch is a device array of
 * T3F_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads it until the
 * process exits. The first call on a device looks up the array's address with that device
 * current (make it before any stream capture). Every call uses the same array, which keeps
 * the previous call's contents; each call clears the error word and overwrites every
 * partial it reads. Calls whose work overlaps on the GPU (e.g. issued on two streams with no
 * ordering between them) race on the array. Returns T3F_ERR_WORKSPACE when a launch would
 * need more scratch than T3F_NOALLOC_SCRATCH_BYTES (a device with more than about 1000
 * SMs). Calls no allocating routine. An out-of-range index is clamped on the device, as in
 * t3f_gather, and recorded in the array's error word: read it with
 * t3f_gather_noalloc_status() after the call (and before the next one on that device).
 */
#define T3F_NOALLOC_SCRATCH_BYTES 65536
t3f_status t3f_gather_noalloc(const t3f_tt* X, const int32_t* idx, int64_t N, const float* y,
                              float* vals, double* loss, t3f_stream_t stream);

/* Device-side status of the last t3f_gather_noalloc call on the current device (the error
 * word of its scratch array): T3F_OK, or T3F_ERR_ARG if an index tuple was out of range.
 * Synchronises `stream`; allocates nothing. */
t3f_status t3f_gather_noalloc_status(t3f_stream_t stream);

/*
 * Adjoint of the gather (paper Section 3.2, Riemannian autodiff, for the completion loss).
 * Weights: w (device float [N]) if non-NULL, else the residual w_t = X(i_t) - y_t (y
 * required; loss, if non-NULL, receives 1/2 sum w_t^2 in FP64).
 *  riemannian == 0: dX (F32, shape of X) = cotangent of sum_t w_t X(i_t):
 *      dX^k[:,i,:] = sum_{t: i_{t,k}=i} w_t l_{t,k-1} (outer) rho_{t,k+1}
 *    (l = prefix row through X's cores, rho = suffix column).
 *  riemannian == 1: X is ignored (may be NULL); U, V are the left-/right-orthogonal forms
 *    from t3f_orthogonalize; X(i_t) is evaluated from V. dX (F32, ranks of U) receives the
 *    tangent coordinates dU_k of P_X(sum_t w_t e_{i_t}): the same scatter with U-prefixes
 *    and V-suffixes, followed by the gauge projection dU_k <- (I - U_k U_k^T) dU_k (k < d).
 */
t3f_status t3f_gather_backward(const t3f_tt* X, const int32_t* idx, int64_t N,
                               const float* w, const float* y, double* loss, t3f_tt* dX,
                               int32_t riemannian, const t3f_tt* U, const t3f_tt* V,
                               void* ws, size_t ws_bytes, t3f_stream_t stream);

/*
 * TT-matrix by TT-vector (paper Section 4, 'matvec'): zip over the batch (C_p = A_p x_p),
 * a batch of 1 on either side broadcasts (Section 3.1). No rounding:
 *   C^k[(a*r_x+b), i, (a'*r_x+b')] = sum_j A^k[a,i,j,a'] x^k[b,j,b'],
 * so C has ranks r^A_k * r^x_k and modes m_k. A: TT-matrix (m != NULL), x: TT-vector with
 * n_k equal to A's column modes; C: F32 TT-vector descriptor of the product's shape.
 * With one column mode 2, 4 or 8 on every core a persistent kernel runs the (pair, core)
 * units, each unit's two cores fetched whole by TMA bulk copies one unit ahead. ws
 * (optional, t3f_workspace_size(T3F_OP_MATVEC) bytes): its error word receives
 * T3F_ERR_TIMEOUT if a copy's bounded wait runs out (see t3f_device_status).
 */
t3f_status t3f_matvec(const t3f_tt* A, const t3f_tt* x, t3f_tt* C, void* ws,
                      size_t ws_bytes, t3f_stream_t stream);

/* Adjoint of t3f_matvec: dA^k[a,i,j,a'] = sum_{b,b'} dC^k[(a,b),i,(a',b')] x^k[b,j,b'],
 * dx^k[b,j,b'] = sum_{a,a',i} dC^k[(a,b),i,(a',b')] A^k[a,i,j,a'] (summed over the batch on
 * a broadcast side). dA or dx may be NULL. ws is not used (may be NULL). */
t3f_status t3f_matvec_backward(const t3f_tt* A, const t3f_tt* x, const t3f_tt* dC,
                               t3f_tt* dA, t3f_tt* dx, void* ws, size_t ws_bytes,
                               t3f_stream_t stream);

/*
 * Ranks after orthogonalisation (host only, integer bookkeeping): right-to-left
 * r'_{k-1} = min(r_{k-1}, n_k r'_k), then left-to-right r''_k = min(r''_{k-1} n_k, r'_k).
 * out_ranks: host [d+1].
 */
t3f_status t3f_orth_ranks(int32_t d, const int32_t* n, const int32_t* ranks,
                          int32_t* out_ranks);

/*
 * Orthogonal forms of X for the tangent space of the fixed-rank manifold (paper
 * Section 3.2): three Householder sweeps in FP64 (right-to-left on X, left-to-right on the
 * result giving U, right-to-left on U giving V), every QR normalised to diag(R) >= 0.
 * U_1..U_{d-1} are left-orthogonal ((r_{k-1} n_k) x r_k unfoldings with orthonormal
 * columns), U_d carries X; V_2..V_d are right-orthogonal, V_1 carries X; full(U) = full(V)
 * = full(X). X: F32 or F64 cores, any batch. U, V: F32 or F64 descriptors of the same
 * batch with ranks t3f_orth_ranks(X). Ranks up to T3F_MAX_RANK, r_{k-1} n_k <= 4096.
 */
t3f_status t3f_orthogonalize(const t3f_tt* X, t3f_tt* U, t3f_tt* V, void* ws,
                             size_t ws_bytes, t3f_stream_t stream);

/*
 * project_sum (paper Section 3.2): tangent coordinates dU of S = P_X(sum_j c_j Z_j),
 * computed as sum_j c_j P_X Z_j:
 *   Zhat_k[:,i,:] = sum_j c_j L^{(j)}_{k-1} Z_j^k[:,i,:] (R^{(j)}_{k+1})^T,
 *   L^{(j)} = left partials of (U, Z_j), R^{(j)} = right partials of (V, Z_j),
 *   dU_k = (I - U_k U_k^T) Zhat_k for k < d (left unfoldings), dU_d = Zhat_d.
 * U, V: F32 orthogonal forms (batch 1); Z: F32 batch with the modes of U; c: device float
 * [Z->batch]; dU: F32 descriptor with U's shape. With Z->batch = 1 and c = 1 this is the
 * projection P_X Z ('project' in Table 1). The TT of S has cores [dU_1, U_1],
 * [[V_k, 0], [dU_k, U_k]], [[V_d], [dU_d]] (ranks <= 2 r).
 * math: FP32 (CUDA cores), or TF32: the U- and V-side contractions of both sweeps
 * (L'_j = sum_i U_i^T (L_j Z_j,i), M = 128 rows of 16 objects x 8, N = r_X, K = r_X n) run on
 * the tensor cores (tcgen05, TF32 operands, FP32 accumulation), the assembly and the gauge
 * projection in FP32; X ranks <= 32, Z ranks <= 8, modes <= 16 and multiples of 8, else
 * T3F_ERR_UNSUPPORTED (also for BF16). A tensor-core wait that runs out writes T3F_ERR_TIMEOUT
 * into the workspace's error word.
 */
t3f_status t3f_project_sum(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z,
                           const float* c, t3f_tt* dU, int32_t math, void* ws,
                           size_t ws_bytes, t3f_stream_t stream);

/*
 * Adjoint of t3f_project_sum with X (U, V) held fixed: given dUbar (F32, U's shape), the
 * cotangent of phi = sum_k <dUbar_k, dU_k>. With W = gauge projection of dUbar and T_W the
 * rank-2r TT of (U, V, W): dc[j] = <T_W, Z_j>, dZ_j = c_j d<T_W, Z_j>/dZ_j. The partial
 * products are recomputed, not taken from the forward call. dZ (F32, Z's shape) or dc
 * (device float [Z->batch]) may be NULL.
 */
t3f_status t3f_project_sum_backward(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z,
                                    const float* c, const t3f_tt* dUbar, t3f_tt* dZ,
                                    float* dc, void* ws, size_t ws_bytes,
                                    t3f_stream_t stream);

/*
 * Batched projection ('project' of the paper's Table 1, Section 3.2, for every object of a
 * batch): dU_j = tangent coordinates of c_j P_X Z_j, without summing over j (c NULL: c_j = 1).
 *   Zhat_j,k[:,i,:] = c_j L^{(j)}_{k-1} Z_j^k[:,i,:] (R^{(j)}_{k+1})^T,
 *   dU_j,k = (I - U_k U_k^T) Zhat_j,k for k < d, dU_j,d = Zhat_j,d.
 * U, V: F32 orthogonal forms (batch 1, ranks <= T3F_MAX_RANK); Z: F32 batch with U's modes;
 * dU: F32 descriptor of batch Z->batch with U's ranks. Summing dU_j over j gives
 * t3f_project_sum's result.
 */
t3f_status t3f_project(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z, const float* c,
                       t3f_tt* dU, void* ws, size_t ws_bytes, t3f_stream_t stream);

/*
 * Gram matrix of tangent vectors of one tangent space (paper Section 3.2, tailored
 * operations): G[a * dB->batch + b] = <xi_a, eta_b> = sum_k <dA_a,k, dB_b,k>, with xi_a, eta_b
 * given by gauge coordinates (outputs of t3f_project / t3f_project_sum at the same X, so the
 * terms of different k are orthogonal). dA, dB: F32 batches of one shape (U's); G: device float
 * [dA->batch][dB->batch]. math: T3F_MATH_FP32 (FP32 CUDA cores, split-K, deterministic
 * reduction) or T3F_MATH_TF32 (tcgen05 TF32 tensor cores fed by TMA, FP32 accumulation; every
 * core block 16-byte aligned with 16-byte-multiple rows, else T3F_ERR_UNSUPPORTED).
 */
t3f_status t3f_tangent_gram(const t3f_tt* dA, const t3f_tt* dB, float* G, int32_t math, void* ws,
                            size_t ws_bytes, t3f_stream_t stream);

/*
 * Projected matrix-by-vector product (paper Section 3.2, P_b(A c)): dU_j = tangent
 * coordinates of P_X (A x_j) for the TT-matrix A (batch 1, or zip with x) and every TT-vector
 * x_j, computed from the Kronecker cores of the product on the fly (the rank r_A r_x TT of
 * A x_j is never formed): left partials of U and right partials of V against A x_j, then
 * Zhat_k = L_{k-1} (A x)_k R_{k+1}^T and the gauge projection. A's row modes equal U's modes,
 * its column modes x's. dU: F32, batch x->batch, U's ranks. Workspace:
 * t3f_project_matvec_workspace_size(U, A, x) bytes.
 */
size_t t3f_project_matvec_workspace_size(const t3f_tt* U, const t3f_tt* A, const t3f_tt* x);
t3f_status t3f_project_matvec(const t3f_tt* U, const t3f_tt* V, const t3f_tt* A, const t3f_tt* x,
                              t3f_tt* dU, void* ws, size_t ws_bytes, t3f_stream_t stream);

/*
 * Linearised Riemannian Hessian of the completion loss applied to a tangent vector (paper
 * Section 3.2, P_X (grad^2 f) P_X Z): for f(X) = 1/2 sum_t (X(i_t) - y_t)^2 the Euclidean
 * Hessian is sum_t e_{i_t} e_{i_t}^T, so out = coordinates of P_X (sum_t xi(i_t) e_{i_t}) for
 * the tangent vector xi with gauge coordinates dZ. xi(i_t) comes from the block recurrence
 * q_k = q_{k-1} V_k + p_{k-1} dZ_k, p_k = p_{k-1} U_k; the scatter is t3f_gather_backward's
 * Riemannian form with those weights. U, V: orthogonal forms (ranks <= 16); idx: device int32
 * [d][N]; dZ, out: F32, U's shape. An out-of-range index is clamped and recorded in the
 * workspace error word.
 */
t3f_status t3f_completion_hvp(const t3f_tt* U, const t3f_tt* V, const int32_t* idx, int64_t N,
                              const t3f_tt* dZ, t3f_tt* out, void* ws, size_t ws_bytes,
                              t3f_stream_t stream);

/*
 * TT rounding (paper Section 3, t3f.round: the approximation of X by a TT of ranks
 * <= max_rank), the TT-SVD recompression in FP64 for every object of the batch: a
 * right-to-left Householder orthogonalisation sweep (diag(R) >= 0), then left to right the
 * SVD of each (r_{k-1} n_k) x r_k unfolding truncated to its leading min(max_rank, .)
 * singular triplets, S V^T pushed into the next core. Every kept left singular vector has its
 * entry of largest magnitude positive (this fixes the cores element by element where the
 * singular values are distinct). X: F32 batch (ranks up to 164 on each QR, every truncated
 * unfolding with min(rows, cols) <= 100, else T3F_ERR_UNSUPPORTED); Y: F32 batch of X's modes
 * with ranks t3f_round_ranks(X, max_rank). ws: t3f_workspace_size(T3F_OP_ROUND, X) bytes.
 */
t3f_status t3f_round_ranks(int32_t d, const int32_t* n, const int32_t* ranks, int32_t max_rank,
                           int32_t* out_ranks);
t3f_status t3f_round(const t3f_tt* X, int32_t max_rank, t3f_tt* Y, void* ws, size_t ws_bytes,
                     t3f_stream_t stream);

/*
 * A ragged collection of TT-vectors: object o has d[o] cores, modes
 * n[noff_o .. noff_o + d[o]) and ranks ranks[roff_o .. roff_o + d[o] + 1), where noff_o and
 * roff_o are the running sums of d and d + 1 over the preceding objects. Its core k is
 * row-major [r_{k-1}][n_k][r_k] and starts at element obj_off[o] + sum_{j<k} r_j n_j r_{j+1}
 * of `cores`. Host arrays are read during the call only.
 */
typedef struct {
  int32_t count;            /* number of objects, >= 1 */
  const int32_t* d;         /* host [count] */
  const int32_t* n;         /* host [sum d] */
  const int32_t* ranks;     /* host [sum (d + 1)], first and last rank of every object 1 */
  const int64_t* obj_off;   /* host [count] element offset of each object's first core */
  void* cores;              /* device */
  int32_t dtype;            /* T3F_F32 or T3F_BF16 */
} t3f_tt_ragged;

/*
 * Gram matrices within groups of a ragged collection (paper Section 4 'gram' / 'norm' over
 * uneven batches, Section 3.1): objects [gstart[g], gstart[g+1]) form group g and must share
 * d and modes; ranks may differ per object (<= T3F_MAX_RANK). Group g's output is the
 * S_g x S_g matrix G_g[a][b] = <X_a, X_b> (local indices, row-major); the groups' matrices
 * are concatenated in `out` (device float). norms (device double [count], nullable) receives
 * sqrt(G_g[a][a]) in FP64.
 * Scheduling: the objects of every group are ordered by rank into buckets {<=8, <=16, <=32,
 * <=64}; tiles[b] (host int32[4], NULL = built-in defaults, each in 1..16) caps the tile side
 * for bucket b. Within a bucket pair, runs of rank-sorted objects grow up to that side while
 * their tile (padded to the run's own largest rank) fits one CTA; the upper triangle of pairs
 * is cut into such tiles, sorted by cost and drained by ONE persistent launch.
 * math (t3f_math): FP32 = CUDA-core FP32 throughout. TF32 (F32 cores) / BF16 (F32 or BF16
 * cores): every pair runs on the tensor cores (operands rounded to TF32 / BF16, FP32
 * accumulation) in tiles of (128/RA) x (128/RB) pairs, RA and RB = 16, 16, 32, 64 for the
 * buckets of the two sides, drained by one persistent launch. A tensor-core wait that runs
 * out writes T3F_ERR_TIMEOUT into the workspace's error word (t3f_device_status).
 * t3f_gram_groups_prepare writes the work list and object tables into `ws` (host-to-device
 * copies; call it once, outside stream capture). t3f_gram_groups and
 * t3f_gram_groups_backward then only launch kernels (memsets + kernels), so they can be
 * captured in a CUDA graph and replayed while X's shapes and `tiles` are unchanged.
 * ws_bytes >= t3f_gram_groups_workspace_size(X, ngroups, gstart, tiles).
 */
size_t t3f_gram_groups_workspace_size(const t3f_tt_ragged* X, int32_t ngroups,
                                      const int32_t* gstart, const int32_t* tiles);
t3f_status t3f_gram_groups_prepare(const t3f_tt_ragged* X, int32_t ngroups,
                                   const int32_t* gstart, const int32_t* tiles, void* ws,
                                   size_t ws_bytes, t3f_stream_t stream);
t3f_status t3f_gram_groups(const t3f_tt_ragged* X, int32_t ngroups, const int32_t* gstart,
                           const int32_t* tiles, int32_t math, float* out, double* norms,
                           void* ws, size_t ws_bytes, t3f_stream_t stream);

/*
 * Adjoint of t3f_gram_groups: dcores (device float, the layout of X's cores with F32
 * elements) receives the cotangent of sum_g sum_ab dout_g[a][b] <X_a, X_b> for the
 * concatenated per-group cotangents dout (device float, like `out`). Every off-diagonal tile
 * uses the symmetrised cotangent dout[a][b] + dout[b][a]. Requires the same prepared `ws`,
 * of at least t3f_gram_groups_backward_workspace_size(..., math) bytes. math (t3f_math):
 *   FP32: CUDA-core FP32 arithmetic: the tiled adjoint drains its own work lists (runs of
 *   rank-sorted objects cut so that a tile's seven partial tiles fit one CTA, side at most 16
 *   whatever `tiles`): tiles that need more than half an SM's shared memory in one
 *   persistent launch of 512-thread CTAs, the rest in a second of 256-thread CTAs, two per SM.
 *   TF32 (F32 cores) / BF16 (F32 or BF16 cores): tensor cores over the forward's tensor-core
 *   tiles: one persistent launch runs every tile's left and right sweeps and stores the
 *   partials of all interfaces after the prepared tables in `ws`; a second drains the
 *   (tile, core, side) gradient items (see t3f_gram_backward). A tensor-core wait that runs
 *   out writes T3F_ERR_TIMEOUT into the workspace's error word.
 */
size_t t3f_gram_groups_backward_workspace_size(const t3f_tt_ragged* X, int32_t ngroups,
                                               const int32_t* gstart, const int32_t* tiles,
                                               int32_t math);
t3f_status t3f_gram_groups_backward(const t3f_tt_ragged* X, int32_t ngroups,
                                    const int32_t* gstart, const int32_t* tiles, int32_t math,
                                    const float* dout, float* dcores, void* ws,
                                    size_t ws_bytes, t3f_stream_t stream);

/*
 * FP32 FMA throughput probe (no counterpart in the paper; a measurement aid for the CUDA-core
 * roofline): `grid` CTAs of 256 threads each run 8 independent FMA chains for iters * 16
 * steps; t3f_fma_probe_flops() gives the FLOPs of one launch. out: device float [grid * 256].
 */
t3f_status t3f_fma_probe(int32_t grid, int64_t iters, float* out, t3f_stream_t stream);
double t3f_fma_probe_flops(int32_t grid, int64_t iters);
/* The same probe in FP64 (the denominator of the FP64 rounding and orthogonalisation);
 * out: device double [grid * 256]. */
t3f_status t3f_fma_probe_f64(int32_t grid, int64_t iters, double* out, t3f_stream_t stream);

/*
 * Device-side error word of the last call that used `ws` (enqueued on `stream`, read after
 * a synchronisation): 0 = none, T3F_ERR_ARG = an index tuple was out of range,
 * T3F_ERR_TIMEOUT = a bounded wait ran out. Synchronises `stream`.
 */
t3f_status t3f_device_status(const void* ws, t3f_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* T3F_H */
