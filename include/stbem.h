/*
 * stbem.h -- C ABI of the GB300 space-time boundary element library for the
 * 2D heat equation  alpha d_t u - Laplace u = 0  (paper: Section 1, eq. (1)).
 *
 * The library covers the data-parallel hot path of the preconditioned
 * space-time Galerkin BEM: assembly of the single layer V_h, double layer K_h
 * and hypersingular D_h matrices on a polygon x uniform time grid
 * (Section 1 eq. (4); Section 2 Theorem), their block-lower-triangular,
 * block-Toeplitz-in-time products (Section 3), the right-hand side
 * (1/2 M_h + K_h) g of eq. (4), and right-preconditioned GMRES with the
 * operator preconditioner C_V^{-1} = M_h^{-1} D_h M_h^{-T} (Section 2, with
 * the lumped mass of Section 4).
 *
 * Conventions (every call):
 *  - Return value: 0 (STBEM_OK) or a negative STBEM_ERR_* code.  No exception
 *    or abort crosses the ABI; stbem_last_error() returns a message for the
 *    last failing call on that context.
 *  - Ownership: every array argument named dev_* is a DEVICE pointer owned by
 *    the caller (e.g. a torch tensor); host_* arrays are host pointers, read
 *    during the call only.  The library allocates only its opaque handles
 *    (a context and meshes, which keep a few KB of geometry on the device).
 *  - Streams: all device work is enqueued on the stream given to
 *    stbem_create() and is asynchronous unless a call says otherwise.
 *  - Layouts: time-major unknowns.  A Toeplitz operator is stored as lag
 *    blocks A[d][i][j], d = 0..n_t-1, row-major, d slowest; it represents the
 *    block matrix whose block (m, n) is A[m-n] for m >= n and 0 otherwise.
 *    Vectors are x[n][j] (n_t x n_cols), batches x[b][n][j].
 *  - Index conventions (geometry): vertices x_0..x_{N-1} counter-clockwise,
 *    segment i = [x_i, x_{i+1 mod N}], outward normal (t_y, -t_x).
 */
#ifndef STBEM_H
#define STBEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define STBEM_OK 0
#define STBEM_ERR_ARG (-1)       /* invalid argument (size, pointer, mesh)   */
#define STBEM_ERR_CUDA (-2)      /* a CUDA runtime call failed               */
#define STBEM_ERR_NOMEM (-3)     /* caller workspace too small               */
#define STBEM_ERR_NOCONV (-4)    /* iteration cap reached before tolerance   */
#define STBEM_ERR_BREAKDOWN (-5) /* GMRES breakdown: a zero Givens pivot,    */
                                 /* i.e. a singular (preconditioned) operator */
#define STBEM_ERR_NAN (-6)       /* NaN or Inf met in a residual             */
#define STBEM_ERR_TIMEOUT (-7)   /* a bounded device-side wait gave up       */
#define STBEM_ERR_REDUCE (-8)    /* the caller's all-reduce callback failed  */

/* operators */
#define STBEM_OP_V 0 /* single layer  <V phi0_k, phi0_l>,   N_x x N_x blocks */
#define STBEM_OP_K 1 /* double layer  <K phi10_p, phi0_i>,  N_x x N_x blocks */
#define STBEM_OP_D 2 /* hypersingular <D psi_k, psi_l>,     N_x x N_x blocks */

/* precisions of stored operators */
#define STBEM_F64 0
#define STBEM_F32 1

typedef struct stbem_ctx stbem_ctx;
typedef struct stbem_mesh stbem_mesh;

/* Create a context on CUDA device `device`; `stream` is a cudaStream_t
 * (NULL = legacy default stream).  Uploads the quadrature tables of the
 * discretisation rule to the device.  Errors: STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_create(stbem_ctx** out, int device, void* stream);
void stbem_destroy(stbem_ctx* ctx);
/* Message of the last failing call on ctx (never NULL). */
const char* stbem_last_error(const stbem_ctx* ctx);
/* Library version string. */
const char* stbem_version(void);
/* Number of CUDA kernels this library has launched in the process (all
 * contexts); a diagnostic counter with no counterpart in the paper. */
unsigned long long stbem_launch_count(void);

/* Measured arithmetic-pipe rates of the context's device (a diagnostic with
 * no counterpart in the paper; the denominators of the rooflines of the
 * ALU-bound kernels): host_out[0] = FP64 FMA TFLOP/s, host_out[1] = FP32 FMA
 * TFLOP/s, host_out[2] = MUFU ex2 results per second in units of 1e12.
 * Independent FMA / ex2 chains on every SM, timed with CUDA events on the
 * context's stream (about 50 ms).  Blocks the host.  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_CUDA. */
int stbem_pipe_peaks(stbem_ctx* ctx, double* host_out);

/* Boundary mesh Gamma_h x I_h (Section 1: tensor-product decomposition of
 * Sigma).  host_xy: 2*n_x doubles (x_0, y_0, x_1, y_1, ...), a closed
 * polygon in counter-clockwise order; n_t uniform steps of length T/n_t; alpha
 * the heat capacity constant.  Errors: STBEM_ERR_ARG if n_x < 3, n_t < 1,
 * T <= 0, alpha <= 0, a segment has zero length or the vertices are clockwise. */
int stbem_mesh_create(stbem_ctx* ctx, const double* host_xy, int n_x, double T,
                      int n_t, double alpha, stbem_mesh** out);
void stbem_mesh_destroy(stbem_mesh* mesh);

/* Bytes of a stored operator: n_t * n_x * n_x * sizeof(element). */
int stbem_op_bytes(const stbem_mesh* mesh, int op, int prec, size_t* bytes);

/* Assemble the lag blocks of op (STBEM_OP_V / K / D) into dev_out
 * (n_t x n_x x n_x, precision prec).  Entries follow the Galerkin
 * definitions of Section 1 eq. (4) (V, K) and the integrated-by-parts form of
 * the hypersingular operator (Section 2, citing Costabel Thm 6.1) on the dual
 * space Y_h (Section 2), integrated by the discretisation rule documented in
 * the repository (Gauss-Legendre in space, graded/Duffy rules for coincident
 * and touching pieces at lags 0-1, closed-form or Peano time integrals).
 * STBEM_F32 is the mixed-precision assembly: FP32 arithmetic and storage,
 * except that identical pieces and pieces sharing a vertex at lags 0 and 1
 * (where the small-argument E1 terms cancel) are integrated in FP64; entries
 * carry about 1e-6 relative error (D_h entries far from the diagonal, which
 * are small differences of larger terms, carry about 1e-6 of their terms).
 * Errors: STBEM_ERR_ARG (bad op/prec/NULL), STBEM_ERR_CUDA. */
int stbem_assemble(stbem_ctx* ctx, const stbem_mesh* mesh, int op, int prec,
                   void* dev_out);

/* The three operators of the boundary integral system (Section 2, eq. (7)):
 * stbem_assemble of V, K and D at once, each into its own n_t x n_x x n_x
 * array of its own precision prec_V / prec_K / prec_D (STBEM_F64 or
 * STBEM_F32, checked for all three; a NULL output is skipped and at least one
 * is given).  D runs on the context's stream and K, V on two side streams the
 * context owns (created on the first call), which wait for the context
 * stream's earlier work and are joined back into it: work enqueued on the
 * context stream afterwards sees all three.  Each operator uses its own slice
 * of the mesh's singular-pair scratch, so the result equals three
 * stbem_assemble calls bit for bit.  Errors as stbem_assemble. */
int stbem_assemble_ops(stbem_ctx* ctx, const stbem_mesh* mesh, int prec_V, int prec_K,
                       int prec_D, void* dev_V, void* dev_K, void* dev_D);

/* As stbem_assemble, restricted to the lag blocks d in [lag_begin, lag_end)
 * (0 <= lag_begin <= lag_end <= n_t); dev_out is still the full
 * n_t x n_x x n_x array and only those blocks are written.  Lag ranges are
 * independent, so a caller can assemble them in pieces, on several streams of
 * different contexts, or shard them across devices.  Calls that include lag
 * 0 or 1 use the mesh's small singular-pair scratch: such calls on one mesh
 * must not overlap in time.  Errors: STBEM_ERR_ARG (bad op, precision or
 * range), STBEM_ERR_CUDA. */
int stbem_assemble_lags(stbem_ctx* ctx, const stbem_mesh* mesh, int op, int prec, int lag_begin,
                        int lag_end, void* dev_out);

/* Block-Toeplitz product (Section 3 block structure).
 *   transpose = 0:  y[b][m][i] = sum_{d=0}^{m} sum_j A[d][i][j] x[b][m-d][j]
 *   transpose = 1:  y[b][n][j] = sum_{d=0}^{n_t-1-n} sum_i A[d][i][j] x[b][n+d][i]
 * A has n_t lag blocks of n_x x n_x in precision prec (F64 or F32); x and y
 * are FP64, n_rhs x n_t x n_x, and must not overlap.  Accumulation is in the
 * precision of A (FP64 for F64, FP32 for F32).  dev_work must hold
 * stbem_apply_workspace_bytes() bytes (partial sums over lag chunks, so the
 * result is deterministic).  The workspace size and the launch shape depend
 * on the SM count of the device that is current when they are computed.
 * Errors: STBEM_ERR_ARG (also when n_rhs times the number of 32-step time
 * tiles exceeds 65535, the grid limit: split the right-hand sides),
 * STBEM_ERR_NOMEM. */
int stbem_apply_workspace_bytes(int n_t, int n_x, int n_rhs, int prec, size_t* bytes);
int stbem_apply(stbem_ctx* ctx, int prec, int transpose, int n_t, int n_x,
                const void* dev_A, int n_rhs, const double* dev_x, double* dev_y,
                void* dev_work, size_t work_bytes);

/* Allocation-free block-Toeplitz product.  The paper has no counterpart: this
 * is a service for callers that cannot allocate device memory at all -- for
 * example code embedded in a host framework that owns every device buffer
 * through its own pool and forbids raw allocations, or a C caller without an
 * allocator -- and so cannot provide the workspace stbem_apply needs.  Same
 * arguments and result as stbem_apply, minus the workspace: the lag-chunk
 * partial sums go to a fixed scratch array inside the library's device image
 * (32 MiB; every GPU that loads the library holds it until the process exits).
 * The first call in each CUDA context of a device looks up that array's device
 * address (after a cudaDeviceReset the next call looks it up again in the new
 * context); make that first call before any stream capture.  Calls share the one array: two calls
 * that overlap on the GPU (other streams, other threads, other contexts on the
 * same device) race on it and must be serialised by the caller.  Each call
 * writes every scratch entry it later reads, so nothing has to start at zero
 * and the previous call's leftovers are never read.  Allocates nothing (no
 * cudaMalloc, no allocating library call).  Errors: STBEM_ERR_ARG (as
 * stbem_apply, including the grid limit on n_rhs);
 * STBEM_ERR_NOMEM if the product needs more scratch than the fixed array
 * holds (stbem_apply_workspace_bytes() > 32 MiB); STBEM_ERR_CUDA. */
int stbem_apply_noalloc(stbem_ctx* ctx, int prec, int transpose, int n_t, int n_x,
                        const void* dev_A, int n_rhs, const double* dev_x, double* dev_y);

/* dev_dst[i] = BF16(dev_src[i]) (round to nearest even), i < n, with src in
 * precision src_prec (STBEM_F64 or STBEM_F32): the operand format of
 * stbem_apply_tc.  Errors: STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_to_bf16(stbem_ctx* ctx, int src_prec, size_t n, const void* dev_src, void* dev_dst);

/* Many-right-hand-side block-Toeplitz product on the tensor cores (Section 3
 * block structure; with n_rhs right-hand sides every lag block multiplies a
 * dense n_x x (n_rhs n_t) matrix):
 *   y[b][m][i] = sum_{d=0}^{m} sum_j A[d][i][j] x[b][m-d][j]
 * A (n_t x n_x x n_x) and x (n_rhs x n_t x n_x) in BF16 (stbem_to_bf16),
 * products accumulated in FP32, y written in FP64 (n_rhs x n_t x n_x).
 * Requires n_x % 8 == 0 and 16-byte aligned A and x.  Blocks the host: it
 * reads the kernel's error word afterwards.  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_TIMEOUT (a pipeline wait gave up; y is incomplete),
 * STBEM_ERR_CUDA. */
int stbem_apply_tc(stbem_ctx* ctx, int n_t, int n_x, const void* dev_A_bf16, int n_rhs, const void* dev_x_bf16,
                   double* dev_y);

/* Diagnostic with no counterpart in the paper: exercises the time-out path of
 * the tensor-core product.  With stall != 0, every later plain tensor-core
 * product (stbem_apply_tc, and those inside stbem_solve_batched; any context)
 * makes its kernel wait on a pipeline barrier that no thread
 * ever arrives on, and every pipeline wait of that kernel gives up after
 * wait_cycles SM clock cycles (>= 1024).  The kernel then lets the tensor-
 * memory operations and copies it has issued complete (each such wait bounded
 * by about one second), releases its tensor memory and exits; the call
 * returns STBEM_ERR_TIMEOUT and y is incomplete.  stall = 0 restores normal
 * operation (wait_cycles is then ignored).  Must not be changed while a
 * tensor-core call is in progress on another thread.  Errors: STBEM_ERR_ARG
 * (stall != 0 with wait_cycles < 1024). */
int stbem_debug_tc_stall(int stall, long long wait_cycles);

/* The same product with compensated accumulation: the tensor cores restart
 * their FP32 accumulator every `chunk` 64-wide K steps (chunk >= 1; one K
 * step is four MMA roundings) and each finished partial is added into a Kahan
 * (sum, compensation) pair per output, so the rounding error no longer grows
 * with the number of lags.  Same arguments, layout and errors as
 * stbem_apply_tc, plus STBEM_ERR_ARG for chunk < 1. */
int stbem_apply_tc_comp(stbem_ctx* ctx, int n_t, int n_x, const void* dev_A_bf16, int n_rhs,
                        const void* dev_x_bf16, double* dev_y, int chunk);

/* Right-hand side of eq. (4) for u_0 = 0 and the Dirichlet datum
 * g = U*(x - y*, t) (y* outside the domain):
 *   dev_g[n][p] = time average of g at vertex p over tau_n,
 *   dev_f       = 1/2 M_h g + K_h g   (M_h of Section 1, K_h given as dev_K).
 * dev_K: the assembled K (FP64); dev_g, dev_f: n_t x n_x doubles; dev_work as
 * for stbem_apply with prec F64, n_rhs = 1. */
int stbem_rhs(stbem_ctx* ctx, const stbem_mesh* mesh, const double* dev_K,
              double y_star_x, double y_star_y, double* dev_g, double* dev_f,
              void* dev_work, size_t work_bytes);

/* Lumped dual mass (Section 4): dev_L[l] = ht (h_{l-1} + 2 h_l + h_{l+1}) / 4,
 * the row sums of M_h[l,k] = <phi0_k, psi_l> (Section 2). n_x doubles. */
int stbem_lumped_mass(stbem_ctx* ctx, const stbem_mesh* mesh, double* dev_L);

/* The consistent mixed mass of Section 2, M_h[l][k] = <phi0_k, psi_l> of one
 * time step (cyclic tridiagonal, not symmetric), inverted on the host by
 * Gauss-Jordan elimination with partial pivoting (N^3 work, once per mesh) and
 * written to dev_Minv (n_x x n_x doubles, row-major).  The paper's Section 4
 * lumps M_h instead (stbem_lumped_mass); with precondition = 2 the solvers use
 * this exact inverse, C_V^{-1} = M_h^{-1} D_h M_h^{-T} as printed in
 * Section 4, which keeps the iteration counts bounded on non-uniform meshes
 * where lumping does not.  Blocks the host.  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_CUDA. */
int stbem_mixed_mass_inverse(stbem_ctx* ctx, const stbem_mesh* mesh, double* dev_Minv);

/* GMRES options and result. */
typedef struct stbem_solve_opts {
  double tol;       /* stop at ||f - V w|| / ||f|| <= tol (paper: 1e-8)     */
  int max_iter;     /* total iteration cap                                 */
  int restart;      /* Krylov dimension before restart                     */
  int precondition; /* 0: none; 1: C_V^{-1} = L^{-1} D_h L^{-1} with the   */
                    /* lumped mass (dev_L: n_x doubles, Section 4); 2:     */
                    /* C_V^{-1} = M_h^{-1} D_h M_h^{-T} (dev_L: n_x x n_x,  */
                    /* stbem_mixed_mass_inverse)                           */
} stbem_solve_opts;

typedef struct stbem_solve_info {
  int iterations;     /* GMRES iterations performed                       */
  int status;         /* STBEM_OK, STBEM_ERR_NOCONV, _BREAKDOWN or _NAN   */
  double rel_residual;/* final true relative residual ||f - V w|| / ||f|| */
} stbem_solve_info;

/* Workspace for stbem_solve: Krylov basis (restart+1 vectors), preconditioned
 * basis, temporaries and product partial sums. */
int stbem_solve_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes);

/* Solve V_h w = f (eq. (4)) by right-preconditioned GMRES (Section 2),
 * x0 = 0, classical Gram-Schmidt with reorthogonalisation in FP64, Givens
 * rotations; the residual tested is the true residual, recomputed at every
 * restart and at the end.  dev_V, dev_D: assembled operators (prec vprec, both
 * the same precision; dev_D and dev_L may be NULL when opts->precondition is
 * 0); dev_L: lumped dual mass (n_x doubles); dev_f, dev_w: n_t x n_x doubles.
 * Blocks the host (reads a residual each iteration).  Returns STBEM_OK,
 * STBEM_ERR_NOCONV (opts->max_iter reached), _BREAKDOWN (a Krylov step gave a
 * zero pivot, so V_h or the preconditioner is singular; w then holds the
 * iterate of the last completed restart cycle) or _NAN (also stored in
 * info->status). */
int stbem_solve(stbem_ctx* ctx, int n_t, int n_x, int vprec, const void* dev_V,
                const void* dev_D, const double* dev_L, const double* dev_f,
                double* dev_w, const stbem_solve_opts* opts, stbem_solve_info* info,
                void* dev_work, size_t work_bytes);

/* Adjoint solve V_h^T lambda = b with the same GMRES and options (the
 * preconditioner becomes L^-1 D_h^T L^-1).  V_h^T is block upper triangular:
 * its product runs backward in time (lambda_n gathers b from steps n + d).
 * Arguments, workspace (stbem_solve_workspace_bytes) and errors as
 * stbem_solve. */
int stbem_solve_adjoint(stbem_ctx* ctx, int n_t, int n_x, int vprec, const void* dev_V,
                        const void* dev_D, const double* dev_L, const double* dev_b,
                        double* dev_lambda, const stbem_solve_opts* opts, stbem_solve_info* info,
                        void* dev_work, size_t work_bytes);

/* ---- Products through time FFTs (Section 3: block lower triangular) -------
 * The product y_n = sum_{d=0}^{n} A_d x_{n-d} with the lag blocks of
 * V_h, K_h or D_h (Toeplitz in time on a uniform grid: the integrals of
 * eq. (4) depend on t - s only) is a convolution in the time index.  With L the smallest
 * power of two >= 2 n_t and w = e^{-2 pi i / L} the frequency blocks are
 *     Ahat_k = sum_{d=0}^{n_t - 1} A_d w^{d k},  k = 0 .. L/2
 * (complex N_x x N_x, stored Ahat[k][i][j] as interleaved (re, im) doubles;
 * the remaining frequencies are their complex conjugates).  A product is a
 * real FFT of x along time, Yhat_k = Ahat_k Xhat_k per frequency, and the
 * inverse real FFT: the same matrix-vector product as stbem_apply up to
 * rounding, with (L/2 + 1) N_x^2 complex multiply-adds in place of
 * n_t (n_t + 1) N_x^2 / 2 real ones and the frequency blocks read once.
 * Rounding: per output row i and right-hand side,
 *     ||y_i - (A x)_i||_2 <= c_L sum_j ||a_ij||_1 ||x_j||_2,
 * a_ij = (A_d[i][j])_d, x_j = (x_n[j])_n, c_L of order log2(L) sqrt(n_t) u
 * (u = 2^-53): a normwise bound, unlike the entrywise one of stbem_apply.
 * Limits: 1 <= n_t <= 4096, 1 <= n_x <= 8192. */

/* Size of the frequency blocks of an n_t x n_x x n_x operator: *n_freq =
 * L/2 + 1 (may be NULL), *bytes = n_freq * n_x * n_x * 16.  Errors:
 * STBEM_ERR_ARG (sizes outside the limits, NULL bytes). */
int stbem_fft_operator_bytes(int n_t, int n_x, int* n_freq, size_t* bytes);

/* dev_Ahat (16-byte aligned, stbem_fft_operator_bytes) from the lag blocks
 * dev_A (n_t x n_x x n_x, FP64 or FP32 by prec; an FP32 operator is widened
 * exactly, which suits a preconditioner such as the mixed D_h).  Errors:
 * STBEM_ERR_ARG (sizes, NULL, alignment, precision), STBEM_ERR_CUDA. */
int stbem_fft_operator(stbem_ctx* ctx, int n_t, int n_x, int prec, const void* dev_A,
                       void* dev_Ahat);

/* Scratch of stbem_apply_fft: the transforms of x and y,
 * 2 n_rhs (L/2 + 1) n_x complex doubles. */
int stbem_apply_fft_workspace_bytes(int n_t, int n_x, int n_rhs, size_t* bytes);

/* dev_y = A dev_x (transpose != 0: A^T x, y_n = sum_d A_d^T x_{n+d}) for
 * n_rhs right-hand sides x[r][n][j] (FP64, n_rhs x n_t x n_x) through the
 * frequency blocks dev_Ahat.  x is read completely before y is written, so
 * dev_y may equal dev_x.  dev_work: 16-byte aligned, at least
 * stbem_apply_fft_workspace_bytes.  Errors: STBEM_ERR_ARG (sizes, NULL,
 * alignment, n_rhs outside [1, 65535]), STBEM_ERR_NOMEM (workspace too
 * small), STBEM_ERR_CUDA. */
int stbem_apply_fft(stbem_ctx* ctx, int transpose, int n_t, int n_x, int n_rhs,
                    const void* dev_Ahat, const double* dev_x, double* dev_y, void* dev_work,
                    size_t work_bytes);

/* Workspace of stbem_solve_fft: that of stbem_solve plus one product's
 * scratch. */
int stbem_solve_fft_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes);

/* stbem_solve (transpose = 0) or stbem_solve_adjoint (transpose != 0) with
 * every product of V_h and D_h taken through their frequency blocks dev_Vhat
 * and dev_Dhat (stbem_fft_operator; dev_Dhat may come from an FP32 D_h: the
 * preconditioner changes the iterations, not the solution).  The GMRES, its
 * options, the FP64 residual test and the errors are those of stbem_solve;
 * dev_work 16-byte aligned, at least stbem_solve_fft_workspace_bytes. */
int stbem_solve_fft(stbem_ctx* ctx, int transpose, int n_t, int n_x, const void* dev_Vhat,
                    const void* dev_Dhat, const double* dev_L, const double* dev_f,
                    double* dev_w, const stbem_solve_opts* opts, stbem_solve_info* info,
                    void* dev_work, size_t work_bytes);

/* ---- Non-uniform time grids (Section 1: any decomposition of (0, T)) ------
 * With time nodes 0 = t_0 < .. < t_{n_t} = T the block of test step m and
 * trial step n <= m depends on (m, n), not on m - n alone: the matrices stay
 * block lower triangular but are not Toeplitz, so all n_t (n_t + 1) / 2
 * blocks are assembled and stored, packed as A[p][i][j] with
 * p = m (m + 1) / 2 + n (N_x x N_x each, FP64).  Time integrals:
 * F(s1) - F(s2) - F(s3) + F(s4), s1 = t_{m+1} - t_n, s2 = t_{m+1} - t_{n+1},
 * s3 = t_m - t_n, s4 = t_m - t_{n+1} (F = 0 for s <= 0), evaluated as on a
 * uniform grid (closed form; the series form with the log terms cancelled at
 * d = m - n = 1; the Peano form over the trapezoid of the overlap length at
 * d >= 2); space rule of the uniform lag d.  Reduces to the Toeplitz blocks
 * on a uniform grid (to rounding).  The rule is stated for neighbouring steps
 * within a ratio of 4. */

/* A boundary mesh on the time nodes host_t[0..n_t] (t_0 = 0, increasing;
 * T = t_{n_t}); otherwise as stbem_mesh_create.  The uniform-grid calls
 * (stbem_assemble, stbem_rhs, ...) reject such a mesh with STBEM_ERR_ARG;
 * every mesh (uniform ones too) can be used with the stbem_nu_* calls. */
int stbem_mesh_create_graded(stbem_ctx* ctx, const double* host_xy, int n_x, const double* host_t, int n_t,
                             double alpha, stbem_mesh** out);
/* Bytes of one packed operator: n_t (n_t + 1) / 2 n_x^2 doubles. */
int stbem_nu_op_bytes(const stbem_mesh* mesh, size_t* bytes);
/* All blocks of op (V, K or D) into dev_out (packed, FP64).  Errors:
 * STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_nu_assemble(stbem_ctx* ctx, const stbem_mesh* mesh, int op, double* dev_out);
/* Block lower-triangular product y[m] = sum_{n <= m} A[p(m, n)] x[n] (x, y:
 * n_t x n_x doubles, not overlapping); every block is read once.  Errors:
 * STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_nu_apply(stbem_ctx* ctx, int n_t, int n_x, const double* dev_A, const double* dev_x, double* dev_y);
/* Right-hand side of eq. (4) for g = U*(x - y*, t), u_0 = 0: dev_g[n][p] the
 * time average of g at vertex p over tau_n, dev_f = 1/2 M_h g + K_h g with
 * M_h[(i,m),(p,m)] = h_m h_i / 2 and the packed dev_K. */
int stbem_nu_rhs(stbem_ctx* ctx, const stbem_mesh* mesh, const double* dev_K, double y_star_x, double y_star_y,
                 double* dev_g, double* dev_f);
/* Lumped dual mass of every step (Section 4 lumping, the step length h_m in
 * place of ht): dev_L[m][l] = h_m (h_{l-1} + 2 h_l + h_{l+1}) / 4. */
int stbem_nu_lumped_mass(stbem_ctx* ctx, const stbem_mesh* mesh, double* dev_L);
/* stbem_solve for packed operators: right-preconditioned GMRES (Section 2
 * preconditioner, opts->precondition = 0 or 1 with dev_L from
 * stbem_nu_lumped_mass).  Workspace: stbem_solve_workspace_bytes.  Errors
 * as stbem_solve. */
int stbem_nu_solve(stbem_ctx* ctx, int n_t, int n_x, const double* dev_V, const double* dev_D, const double* dev_L,
                   const double* dev_f, double* dev_w, const stbem_solve_opts* opts, stbem_solve_info* info,
                   void* dev_work, size_t work_bytes);

/* ---- Lag sharding of one problem across ranks (Section 3) -------------------
 * The paper distributes the blocks of its block-lower-triangular matrices over
 * processes.  On a uniform time grid all blocks at one lag are equal, so here
 * the lag block is the unit: a rank holds the blocks of some lags, computes
 * its part of every product, y_r[m] = sum_{d held} A^(d) x[m - d], and one
 * sum over ranks (an all-reduce of n_t x n_x doubles) completes the product.
 * Vectors, the right-hand side, the preconditioner's masses and the GMRES
 * recurrences are replicated on every rank; only the operators are split. */

/* Lag ranges of `rank` among n_ranks: chunks of `chunk` consecutive lags dealt
 * in snake order (0, 1, .., R-1, R-1, .., 0, 0, ..), so that the work
 * sum (n_t - d) and the number of blocks balance across ranks; adjacent chunks
 * of one rank are merged.  host_ranges receives 2 * (*n_ranges) ints
 * [begin, end) in increasing order; *n_ranges may be 0 (more ranks than
 * chunks).  Host only, no device needed.  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_NOMEM (*n_ranges > max_ranges; *n_ranges tells how many). */
int stbem_lag_shard(int n_t, int n_ranks, int rank, int chunk, int max_ranges, int* host_ranges, int* n_ranges);

/* As stbem_assemble_lags, but the blocks of the lags [lag_begin, lag_end) are
 * written compactly: block d to dev_blocks + (d - lag_begin) n_x^2 elements
 * (dev_blocks holds (lag_end - lag_begin) n_x^2 elements).  Errors as
 * stbem_assemble_lags. */
int stbem_assemble_lag_blocks(stbem_ctx* ctx, const stbem_mesh* mesh, int op, int prec, int lag_begin, int lag_end,
                              void* dev_blocks);

/* The block-Toeplitz product restricted to the lags [lag_begin, lag_end):
 *   transpose = 0: y[b][m] (=, or += with accumulate) sum_{d in range, d <= m} A^(d) x[b][m-d]
 *   transpose = 1: y[b][n] (=, or +=) sum_{d in range, n + d < n_t} A^(d)^T x[b][n+d]
 * with dev_A_blocks holding those blocks compactly (block d at
 * (d - lag_begin) n_x^2).  Accumulation, layouts and workspace
 * (stbem_apply_lags_workspace_bytes with n_lags = lag_end - lag_begin) as
 * stbem_apply.  Errors as stbem_apply. */
int stbem_apply_lags_workspace_bytes(int n_t, int n_x, int n_lags, int n_rhs, size_t* bytes);
int stbem_apply_lags(stbem_ctx* ctx, int prec, int transpose, int n_t, int n_x, int lag_begin, int lag_end,
                     const void* dev_A_blocks, int n_rhs, const double* dev_x, double* dev_y, int accumulate,
                     void* dev_work, size_t work_bytes);

/* All-reduce (sum over ranks, in place) of n doubles at dev_buf, supplied by
 * the caller (e.g. NCCL or gloo through torch.distributed).  It is called on
 * the host after this rank's partial product has been enqueued on the
 * context's stream; it must sum over ranks what that stream has produced and
 * leave the result in dev_buf before later work on the stream reads it (for
 * a collective on another stream: make it wait for the context's stream, and
 * the context's stream for it).  Returns 0 on success. */
typedef int (*stbem_allreduce_fn)(double* dev_buf, size_t n, void* user);

/* Lag-sharded stbem_solve: the same right-preconditioned GMRES on every rank,
 * whose V and D products are the rank's lag ranges (stbem_lag_shard;
 * host_ranges, n_ranges, the same for V and D) of the compact operators
 * dev_V_blocks and dev_D_blocks, followed by allreduce(y, n_t n_x, user).
 * Every rank must call it with the same f, L and options; all ranks then
 * perform the same iterations and return the same w.  A rank holding no lags
 * passes n_ranges = 0 (its partial products are zero).  Workspace:
 * stbem_solve_sharded_workspace_bytes.  Errors as stbem_solve, and
 * STBEM_ERR_REDUCE when the callback returns non-zero (the solve stops). */
int stbem_solve_sharded_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes);
int stbem_solve_sharded(stbem_ctx* ctx, int n_t, int n_x, int vprec, const void* dev_V_blocks,
                        const void* dev_D_blocks, int n_ranges, const int* host_ranges, stbem_allreduce_fn allreduce,
                        void* user, const double* dev_L, const double* dev_f, double* dev_w,
                        const stbem_solve_opts* opts, stbem_solve_info* info, void* dev_work, size_t work_bytes);

/* Shape and alpha gradient by the adjoint method (not in the paper, which
 * does not differentiate; it differentiates the discrete system of eq. (4)).
 * For w solving V_h w = f, f = 1/2 M_h g + K_h g with g the time averages of
 * U*(x - y*, t) at the vertices (stbem_rhs), and lambda solving
 * V_h^T lambda = dL/dw (stbem_solve_adjoint), writes
 *   dev_dxy[2 k + c] = lambda^T (df/dx_k,c - (dV_h/dx_k,c) w)   (n_x x 2 doubles)
 *   dev_dalpha[0]    = lambda^T (df/dalpha - (dV_h/dalpha) w),
 * the derivatives of L with respect to the polygon vertices and alpha.  The
 * derivatives of V_h and K_h are recomputed tile by tile from the quadrature
 * of the assembly (same rule, derivative of the integrand) and contracted with
 * C(d) = sum_m lambda_m x_{m-d}^T (x = w for V_h, g for K_h); nothing of size
 * n_t n_x^2 n_params is stored.  dev_K: the assembled K (FP64); dev_g, dev_w,
 * dev_lambda: n_t x n_x doubles.  FP64 throughout.  Workspace:
 * stbem_grad_workspace_bytes() (two n_t n_x^2 correlation arrays and per-pair
 * partial sums), 256-byte aligned.  Asynchronous on the context's stream.
 * Errors: STBEM_ERR_ARG, STBEM_ERR_NOMEM, STBEM_ERR_CUDA. */
int stbem_grad_workspace_bytes(int n_t, int n_x, size_t* bytes);
int stbem_grad(stbem_ctx* ctx, const stbem_mesh* mesh, const double* dev_K, double y_star_x,
               double y_star_y, const double* dev_g, const double* dev_w, const double* dev_lambda,
               double* dev_dxy, double* dev_dalpha, void* dev_work, size_t work_bytes);

/* Mixed-precision solve of V_h w = f (eq. (4)): FP64 iterative refinement,
 * r = f - V_h w with the FP64 operator dev_V64, around right-preconditioned
 * GMRES (Section 2 preconditioner) on the FP32 operators dev_V32 and dev_D32
 * (FP32 products, FP64 Krylov vectors and orthogonalisation).  Each inner
 * solve reduces its residual by inner_tol (0 < inner_tol < 1, e.g. 1e-4);
 * refinement stops when the FP64 residual ||f - V64 w|| / ||f|| <= opts->tol.
 * opts->max_iter caps the inner iterations in total; info->iterations reports
 * them.  Workspace: stbem_solve_mixed_workspace_bytes().  Errors as
 * stbem_solve. */
int stbem_solve_mixed_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes);
int stbem_solve_mixed(stbem_ctx* ctx, int n_t, int n_x, const double* dev_V64, const float* dev_V32,
                      const float* dev_D32, const double* dev_L, const double* dev_f, double* dev_w,
                      const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* info,
                      void* dev_work, size_t work_bytes);

/* dev_dst[i] = (float)dev_src[i], i < n (rounds an FP64 operator to FP32 for
 * the inner solves of stbem_solve_mixed; a utility with no counterpart in the
 * paper).  Errors: STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_round_f32(stbem_ctx* ctx, size_t n, const double* dev_src, float* dev_dst);

/* Three-term BF16 split of an FP64 array: hi = BF16(x), mid = BF16(x - hi),
 * lo = BF16(x - hi - mid) (mid and lo may be NULL), so that
 * |x - (hi + mid + lo)| <= ~2^-24 |x|.  Operand format of stbem_apply_tc3 and
 * stbem_solve_batched.  Errors: STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_bf16_split3(stbem_ctx* ctx, size_t n, const double* dev_src, void* dev_hi, void* dev_mid, void* dev_lo);

/* Accurate many-right-hand-side product on the tensor cores: with A given by
 * its three BF16 slices (stbem_bf16_split3; dev_A_mid / dev_A_lo may be NULL)
 * and x (FP64) split the same way inside the call, y = sum of the six slice
 * products A_s x_t with s + t <= 2, each with the compensated accumulation of
 * stbem_apply_tc_comp (partials of 4 K steps for hi x hi, 16 for the rest),
 * summed in FP64: a few 1e-7 relative to |A| |x|, against ~4e-3 for one BF16
 * product and ~4e-4 for the uncompensated split product over 512 lags.  Workspace: stbem_apply_tc3_workspace_bytes() (the three
 * slices of x and, with few output tiles, the partial products of chunks of
 * 64 lags per tile), 256-byte aligned.  Blocks the host.  Errors as
 * stbem_apply_tc, STBEM_ERR_NOMEM. */
int stbem_apply_tc3_workspace_bytes(int n_t, int n_x, int n_rhs, size_t* bytes);
int stbem_apply_tc3(stbem_ctx* ctx, int n_t, int n_x, const void* dev_A_hi, const void* dev_A_mid,
                    const void* dev_A_lo, int n_rhs, const double* dev_x, double* dev_y, void* dev_work,
                    size_t work_bytes);

/* ---- Tuned launch parameters ---------------------------------------------------
 * A process-wide table of tuned launch parameters (the plain tensor-core
 * product's tile width, the ragged product's tile family and lag-chunk
 * length), keyed by "device|kernel|shape" strings with "name=value" values,
 * optionally mirrored to a text file ("key<TAB>value" lines after a header;
 * rewritten whole through a temporary file on every store) so that a later
 * process reuses earlier measurements.  The STBEM_TUNE_CACHE environment
 * variable names the default file.  These calls make no CUDA call.
 * stbem_tune_cache_path: NULL or "" keeps the table in memory only; otherwise
 * the file's entries are merged in (a missing file is an empty table;
 * STBEM_ERR_ARG if it exists but cannot be read).
 * stbem_tune_cache_get: STBEM_OK and the value (NUL-terminated) in host_value,
 * STBEM_ERR_ARG if the key is absent, STBEM_ERR_NOMEM if cap is too small.
 * stbem_tune_cache_put: keys and values must be non-empty with no tabs or line
 * breaks (else STBEM_ERR_ARG, also when the file cannot be written).
 * stbem_tune_cache_clear: drops the in-process entries, not the file's. */
int stbem_tune_cache_path(const char* path);
int stbem_tune_cache_get(const char* key, char* host_value, size_t cap);
int stbem_tune_cache_put(const char* key, const char* value);
int stbem_tune_cache_clear(void);

/* Tile-width tuner of the plain tensor-core product (stbem_apply_tc, and the
 * products inside stbem_solve_batched): times 128 x 128 and 128 x 256 output
 * tiles (steps per tile; 256 only when n_t > 128) on this shape (A, x, y as in
 * stbem_apply_tc; y is overwritten) and records the faster in the tune cache,
 * which every later product of the same (n_t, n_x, n_rhs) on this device
 * consults; untuned shapes take 256 for n_t > 128.  With a cached entry the
 * call only reports it (*from_cache = 1).  tile_n, from_cache may be NULL.
 * Blocks the host.  Errors as stbem_apply_tc, and STBEM_ERR_ARG when the
 * cache file cannot be written. */
int stbem_tc_tune(stbem_ctx* ctx, int n_t, int n_x, const void* dev_A_bf16, int n_rhs, const void* dev_x_bf16,
                  double* dev_y, int* tile_n, int* from_cache);

/* ---- Exact-slice products (FP64-grade accuracy on the BF16 tensor cores) -----
 * The block-Toeplitz product of eq. (5)'s lag blocks with many right-hand
 * sides, y[b][m] = sum_{d <= m} A[d] x[b][m - d] (the product the GMRES of
 * Section 2 repeats), computed from integer slices: each row r of an FP64
 * matrix (a row i of a lag block A[d], or the values x[b][n][.] of one step)
 * gets a power-of-two scale 2^e_r (max |row| < 2^e_r) and n_slices signed
 * integer slices q_s of 6 bits, row = 2^e_r sum_s q_s 2^{-6 (s + 1)}
 * (|q_0| <= 64, |q_s| <= 32 after), stored as BF16 (exact).  The product
 * multiplies every slice pair (s, t) with s + t < n_slices on the tensor
 * cores; the integer sums of one lag, one s + t and at most 1024 columns are
 * exact in the FP32 accumulator, and they are combined in double-float with
 * their powers of two, so the only errors are the truncated slice tails and
 * the dropped pairs, relative to the row scales:
 *   |y[b][m][i] - (A x)[b][m][i]|
 *     <= 2^(-6 n_slices) (1 + n_slices / 4) n_x sum_d 2^(eA[d][i] + eX[b][m-d]).
 * Rows whose entries span many decades (the early time steps of a density
 * with a distant source) keep this accuracy relative to their maxima only.
 * Normwise the product is accurate to a few 1e-13 at n_slices = 7 on the
 * batched heat problem (versus ~1e-7 for stbem_apply_tc3 and ~4e-3 for one
 * BF16 product).  Contributions more than 2^-125 below
 * 2^(max_d eA[d][i] + max_{n <= m} eX[b][n]) are dropped.  n_slices is 4..8. */
typedef struct stbem_exact_operand {
  int n_slices;         /* 4..8 */
  const void* slices;   /* device, BF16 [n_slices][rows][cols], 16-byte aligned */
  const int* row_exp;   /* device, int32 [rows]: e_r (-16384 for a zero row) */
} stbem_exact_operand;

/* Slices of an FP64 row-major matrix dev_src (rows x cols) into dev_slices
 * (BF16 [n_slices][rows][cols]) and dev_row_exp (int32 [rows]).  For lag
 * blocks rows = n_t n_x, cols = n_x; for right-hand sides rows = n_rhs n_t,
 * cols = n_x.  Asynchronous on the context's stream.  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_CUDA. */
int stbem_exact_slices(stbem_ctx* ctx, long long rows, int cols, int n_slices, const double* dev_src,
                       void* dev_slices, int* dev_row_exp);

/* y (FP64, [n_rhs][n_t][n_x]) = the block-Toeplitz product of the sliced lag
 * blocks A (rows n_t n_x) with the sliced right-hand sides x (rows n_rhs n_t),
 * both with the same n_slices.  Requires n_x % 8 == 0, n_t <= 4096,
 * n_rhs <= 65535.  One launch of 128 x 128 output tiles; its pipeline waits
 * are bounded (STBEM_ERR_TIMEOUT).  Blocks the host.  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_TIMEOUT, STBEM_ERR_CUDA. */
int stbem_apply_tc_exact(stbem_ctx* ctx, int n_t, int n_x, const stbem_exact_operand* A, int n_rhs,
                         const stbem_exact_operand* x, double* dev_y);

/* The same product with x in FP64 ([n_rhs][n_t][n_x]), sliced inside the call
 * into dev_work (stbem_apply_exact_workspace_bytes(), 256-byte aligned).  When
 * the output tiles are too few to fill the GPU (small n_rhs) the workspace
 * also holds partial products of chunks of 64 lags per tile, summed in chunk
 * order afterwards.  Blocks the host.  Errors as stbem_apply_tc_exact,
 * STBEM_ERR_NOMEM. */
int stbem_apply_exact_workspace_bytes(int n_t, int n_x, int n_rhs, int n_slices, size_t* bytes);
int stbem_apply_exact(stbem_ctx* ctx, int n_t, int n_x, const stbem_exact_operand* A, int n_rhs,
                      const double* dev_x, double* dev_y, void* dev_work, size_t work_bytes);

/* Time averages of g = U*(x - y_k*, t) at the vertices for n_src source
 * points (host_ystar: 2 n_src doubles): dev_G[k][n][p] as in stbem_rhs. */
int stbem_rhs_g_batched(stbem_ctx* ctx, const stbem_mesh* mesh, int n_src, const double* host_ystar,
                        double* dev_G);

/* dev_F[b] += 1/2 M_h dev_G[b] for n_rhs right-hand sides (M_h of eq. (4)). */
int stbem_half_mass_add(stbem_ctx* ctx, const stbem_mesh* mesh, int n_rhs, const double* dev_G, double* dev_F);

/* Solve V_h W_b = F_b for n_rhs right-hand sides at once (the batched form of
 * the Section 2 GMRES): lockstep right-preconditioned GMRES on the BF16 V
 * (dev_V_hi) with the BF16 preconditioner dev_D_bf16 (Section 2, Section 4
 * lumping, dev_L), both applied on the tensor cores, FP64 Krylov vectors and
 * orthogonalisation, a Hessenberg matrix and a convergence mask per
 * right-hand side; each inner solve reduces its residual by inner_tol.  Around
 * it, refinement with the residual R = F - V W from the three-slice split of V
 * (dev_V_hi/mid/lo); that product is accurate to a few 1e-7 of |V||W|, which
 * limits attainable residuals to ~1e-6.  With dev_V64 (the FP64 operator, may
 * be NULL) refinement continues, once every relative residual is below 2e-6,
 * on the FP64 residual F - V64 W (CUDA-core FP64 product of all right-hand
 * sides), so that ||R_b|| / ||F_b|| <= opts->tol holds for the FP64 operator
 * and the solutions carry FP64-solve accuracy; without it the stop is on the
 * split residual.  opts->restart is the Krylov dimension of an inner solve,
 * opts->max_iter caps inner iterations.  infos: n_rhs results (rel_residual:
 * the last residual tested).  Workspace: stbem_solve_batched_workspace_bytes()
 * with fp64_residual != 0 when dev_V64 is given (it then adds the FP64
 * product's partial sums).  Requires n_x % 8 == 0.  Blocks the host.  Errors:
 * STBEM_ERR_ARG, STBEM_ERR_NOMEM, STBEM_ERR_NOCONV / _NAN / _BREAKDOWN (some
 * right-hand side; see infos), STBEM_ERR_TIMEOUT, STBEM_ERR_CUDA. */
int stbem_solve_batched_workspace_bytes(int n_t, int n_x, int n_rhs, int restart, int fp64_residual, size_t* bytes);
int stbem_solve_batched(stbem_ctx* ctx, int n_t, int n_x, int n_rhs, const void* dev_V_hi, const void* dev_V_mid,
                        const void* dev_V_lo, const void* dev_D_bf16, const double* dev_L, const double* dev_V64,
                        const double* dev_F, double* dev_W, const stbem_solve_opts* opts, double inner_tol,
                        stbem_solve_info* infos, void* dev_work, size_t work_bytes);

/* stbem_solve_batched with the exact-slice operator V_exact (stbem_exact_slices
 * of the FP64 V) in place of dev_V64: once every relative residual is below
 * 2e-6, refinement continues on F - V W from the exact-slice product (normwise
 * a few 1e-13 at n_slices = 7; see stbem_exact_operand) on the tensor cores
 * instead of the FP64 CUDA-core product.  Workspace:
 * stbem_solve_batched_exact_workspace_bytes() (the base workspace plus the
 * slices of W), 256-byte aligned.  Requires, besides the sizes of
 * stbem_solve_batched, n_t <= 4096.  Errors as stbem_solve_batched. */
int stbem_solve_batched_exact_workspace_bytes(int n_t, int n_x, int n_rhs, int restart, int n_slices,
                                              size_t* bytes);
int stbem_solve_batched_exact(stbem_ctx* ctx, int n_t, int n_x, int n_rhs, const void* dev_V_hi,
                              const void* dev_V_mid, const void* dev_V_lo, const void* dev_D_bf16,
                              const double* dev_L, const stbem_exact_operand* V_exact, const double* dev_F,
                              double* dev_W, const stbem_solve_opts* opts, double inner_tol,
                              stbem_solve_info* infos, void* dev_work, size_t work_bytes);

/* stbem_solve_batched with the frequency blocks dev_Vhat of the FP64 V
 * (stbem_fft_operator) in place of dev_V64: once every relative residual is
 * below 2e-6, refinement continues on F - V W from the product through time
 * FFTs of all right-hand sides (FP64, normwise; see stbem_apply_fft).
 * Workspace: stbem_solve_batched_fft_workspace_bytes() (the base workspace
 * plus the transforms of W and of V W), 256-byte aligned; dev_Vhat 16-byte
 * aligned.  Requires, besides the sizes of stbem_solve_batched, the limits
 * of stbem_apply_fft.  Errors as stbem_solve_batched. */
int stbem_solve_batched_fft_workspace_bytes(int n_t, int n_x, int n_rhs, int restart, size_t* bytes);
int stbem_solve_batched_fft(stbem_ctx* ctx, int n_t, int n_x, int n_rhs, const void* dev_V_hi,
                            const void* dev_V_mid, const void* dev_V_lo, const void* dev_D_bf16,
                            const double* dev_L, const void* dev_Vhat, const double* dev_F,
                            double* dev_W, const stbem_solve_opts* opts, double inner_tol,
                            stbem_solve_info* infos, void* dev_work, size_t work_bytes);

/* stbem_solve_mixed with the exact-slice operator V_exact (stbem_exact_slices
 * of the FP64 V) in place of dev_V64: every outer residual f - V w is the
 * exact-slice tensor-core product (normwise a few 1e-13 at n_slices = 7; see
 * stbem_exact_operand) instead of the FP64 CUDA-core product.  The FP64 V
 * itself is not needed.  Workspace: stbem_solve_mixed_exact_workspace_bytes()
 * (the mixed solve's plus the slices of w), 256-byte aligned.  Requires
 * n_x % 8 == 0 and n_t <= 4096.  Errors as stbem_solve_mixed, and
 * STBEM_ERR_TIMEOUT. */
int stbem_solve_mixed_exact_workspace_bytes(int n_t, int n_x, int restart, int n_slices, size_t* bytes);
int stbem_solve_mixed_exact(stbem_ctx* ctx, int n_t, int n_x, const stbem_exact_operand* V_exact,
                            const float* dev_V32, const float* dev_D32, const double* dev_L, const double* dev_f,
                            double* dev_w, const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* info,
                            void* dev_work, size_t work_bytes);

/* stbem_solve_mixed_exact with the inner GMRES on the BF16 tensor cores: V and
 * D given by their three BF16 slices (stbem_bf16_split3 of the FP64 V and D;
 * dev_*_mid / dev_*_lo may be NULL), every inner product the compensated
 * three-slice product of stbem_apply_tc3 (a few 1e-7 of |A| |x|, the accuracy
 * of an FP32 product), the outer residuals exact-slice products of V_exact.
 * With few output tiles the products split each tile's lags into chunks.
 * Preconditioner as stbem_solve_mixed (opts->precondition 1: lumped, 2: the
 * consistent mixed mass inverse).  Workspace:
 * stbem_solve_mixed_tc_workspace_bytes(), 256-byte aligned.  Requires
 * n_x % 8 == 0, n_t <= 4096.  Errors as stbem_solve_mixed_exact. */
int stbem_solve_mixed_tc_workspace_bytes(int n_t, int n_x, int restart, int n_slices, size_t* bytes);
int stbem_solve_mixed_tc(stbem_ctx* ctx, int n_t, int n_x, const stbem_exact_operand* V_exact,
                         const void* dev_V_hi, const void* dev_V_mid, const void* dev_V_lo, const void* dev_D_hi,
                         const void* dev_D_mid, const void* dev_D_lo, const double* dev_L, const double* dev_f,
                         double* dev_w, const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* info,
                         void* dev_work, size_t work_bytes);

/* ---- Ragged batches ----------------------------------------------------------
 * Many independent problems of different sizes (not in the paper, which solves
 * one problem at a time): every problem has its own polygon, N_x, N_t, T and
 * alpha.  The batch handle owns the problems' meshes and the work lists of the
 * persistent launches.  Batch arrays are the problems' arrays concatenated in
 * problem order (stbem_ragged_offsets gives the start of each):
 *   operators  sum_p n_t N_x^2 elements (A_p[d][i][j] as for one problem),
 *   vectors    sum_p n_t N_x doubles   (x_p[n][j]),
 *   masses     sum_p N_x doubles.
 * All device arrays are caller-owned. */
typedef struct stbem_ragged stbem_ragged;
typedef struct stbem_problem {
  const double* xy;   /* host: 2 n_x vertex coordinates, counter-clockwise */
  int n_x, n_t;
  double T, alpha;
} stbem_problem;

/* Builds every problem's mesh (errors as stbem_mesh_create). */
int stbem_ragged_create(stbem_ctx* ctx, int n_problems, const stbem_problem* problems, stbem_ragged** out);
void stbem_ragged_destroy(stbem_ragged* batch);
int stbem_ragged_sizes(const stbem_ragged* batch, long long* op_elems, long long* vec_elems, long long* mass_elems);
/* start offsets (elements) of each problem: host arrays of n_problems (any may be NULL) */
int stbem_ragged_offsets(const stbem_ragged* batch, long long* op_off, long long* vec_off, long long* mass_off);

/* Lag blocks of op (STBEM_OP_V, K or D, Section 1 eq. (4) / Section 2) for
 * every problem, precision prec (F64 or F32 as stbem_assemble): one persistent
 * launch over the lag-0/1 identical and vertex-sharing pairs of all problems,
 * then one over all (problem, lag, tile) items, largest problems first.
 * Asynchronous. */
int stbem_ragged_assemble(stbem_ctx* ctx, stbem_ragged* batch, int op, int prec, void* dev_out);
/* lumped dual mass (Section 4) of every problem into the masses array */
int stbem_ragged_lumped_mass(stbem_ctx* ctx, stbem_ragged* batch, double* dev_L);

/* y_p = A_p x_p for every problem (Section 3 block-Toeplitz product): one
 * persistent launch over all (problem, lag chunk, time tile, row tile) units
 * and one reduction.  Workspace: stbem_ragged_apply_workspace_bytes (enough
 * for every lag-chunk length the tuner tries).  Asynchronous. */
int stbem_ragged_apply_workspace_bytes(const stbem_ragged* batch, size_t* bytes);
int stbem_ragged_apply(stbem_ctx* ctx, stbem_ragged* batch, int prec, const void* dev_A, const double* dev_x,
                       double* dev_y, void* dev_work, size_t work_bytes);
/* Autotuner: times the product with A (dev_x, dev_y: batch vectors used as
 * input and output) with CUDA events for each candidate tile family (FP32
 * products: the register-tiled kernel, which needs every N_x % 4 == 0, and
 * the generic tiles; FP64: the generic tiles) and lag-chunk length (32 .. 512
 * lags per partial), and keeps the fastest for every later product and solve
 * of this batch.  The choice is recorded in the tune cache (stbem_tune_cache_*)
 * under the device, the precision and the batch's (N_x, N_t) list; when the
 * cache already holds an entry for them the call applies it without timing.
 * lags_per_chunk / tiles32 (may be NULL) receive the choice.  Blocks the host.
 * stbem_ragged_tune_report returns the candidates timed by the last call
 * (lag-chunk length, tile family 1 = register tiles, time in ms; none when the
 * choice came from the cache, *from_cache = 1). */
int stbem_ragged_tune(stbem_ctx* ctx, stbem_ragged* batch, int prec, const void* dev_A, const double* dev_x,
                      double* dev_y, void* dev_work, size_t work_bytes, int* lags_per_chunk, int* tiles32);
int stbem_ragged_tune_report(const stbem_ragged* batch, int max_n, int* candidates, int* tiles32, float* ms,
                             int* n_out, int* from_cache);

/* Right-hand sides of eq. (4) for every problem, g = U*(x - y_p*, t) with the
 * source host_ystar[2p], [2p+1]: dev_g (vertex time averages) and
 * dev_f = 1/2 M_h g + K_h g (dev_K of precision kprec).  Workspace: 256 bytes
 * plus stbem_ragged_apply_workspace_bytes.  Blocks the host. */
int stbem_ragged_rhs(stbem_ctx* ctx, stbem_ragged* batch, int kprec, const void* dev_K, const double* host_ystar,
                     double* dev_g, double* dev_f, void* dev_work, size_t work_bytes);

/* V_p w_p = f_p for every problem: right-preconditioned GMRES (Section 2
 * preconditioner) in lockstep, per-problem Hessenberg and convergence, the
 * device part of each Arnoldi step captured once as a CUDA graph and
 * replayed.  Operators of precision prec (F64 or F32), FP64 vectors; each
 * problem stops at its true relative residual <= opts->tol.  infos: one per
 * problem.  Blocks the host.  Errors as stbem_solve. */
int stbem_ragged_solve_workspace_bytes(const stbem_ragged* batch, int restart, size_t* bytes);
int stbem_ragged_solve(stbem_ctx* ctx, stbem_ragged* batch, int prec, const void* dev_V, const void* dev_D,
                       const double* dev_L, const double* dev_f, double* dev_w, const stbem_solve_opts* opts,
                       stbem_solve_info* infos, void* dev_work, size_t work_bytes);

/* V_p w_p = f_p for every problem to FP64 accuracy with FP32 inner solves
 * (the batched counterpart of stbem_solve_mixed): FP64 iterative refinement,
 * r_p = f_p - V64_p w_p with the FP64 operators dev_V64, around the lockstep
 * solve of stbem_ragged_solve on the FP32 operators dev_V32 (and dev_D32 with
 * the lumped masses dev_L as preconditioner, opts->precondition = 1; NULL D32
 * and precondition = 0 for none), each inner solve reducing its residual by
 * inner_tol (0 < inner_tol < 1).  A problem stops once its FP64 residual
 * ||r_p|| / ||f_p|| <= opts->tol; its later corrections are not computed.
 * opts->max_iter caps the inner iterations (lockstep count); infos[p]
 * reports each problem's inner iterations and final FP64 residual.
 * Workspace: stbem_ragged_solve_mixed_workspace_bytes.  Blocks the host.
 * Errors as stbem_ragged_solve. */
int stbem_ragged_solve_mixed_workspace_bytes(const stbem_ragged* batch, int restart, size_t* bytes);
int stbem_ragged_solve_mixed(stbem_ctx* ctx, stbem_ragged* batch, const double* dev_V64, const float* dev_V32,
                             const float* dev_D32, const double* dev_L, const double* dev_f, double* dev_w,
                             const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* infos, void* dev_work,
                             size_t work_bytes);

/* ---- Initial datum (Section 1, eq. (4): M_h^0 u_0) ------------------------
 * The initial datum u_0 is discretised in S_h^1(Omega_h), the continuous
 * piecewise linear functions on a triangulation of the domain, and
 *   M_h^0[(m,i), j] = int_{tau_m} int_{gamma_i} int_Omega U*(x - y, t) phi_j(y) dy ds_x dt
 * (U* the fundamental solution of Section 1, no 1/alpha factor); the
 * right-hand side of eq. (4) is (1/2 M_h + K_h) g - M_h^0 u_0.  The time
 * integral is exact (differences of alpha/(4 pi) E1(alpha r^2 / (4 t)) at
 * t_m, t_{m+1}); space by the repository's rule per (segment, triangle) pair:
 * tensor Gauss rules whose order depends on the pair class (touching / near /
 * regular) and on m, a polar rule with a sinh transformation for touching
 * pairs at m = 0.  Entries are stored dense as M0[m][i][j] (m slowest). */
typedef struct stbem_domain stbem_domain;

/* Triangulation Omega_h of the domain bounded by mesh.  host_nodes: 2*n_nodes
 * doubles (x, y pairs); host_tris: 3*n_tris node indices, every triangle
 * counter-clockwise with positive area.  Every vertex of mesh must coincide
 * (within 1e-12 of the nodes' bounding-box size) with a node, which is then
 * moved onto the vertex exactly.  The mesh must outlive the domain.  Errors:
 * STBEM_ERR_ARG (NULL, too few nodes/triangles, index out of range, a
 * clockwise or degenerate triangle, a vertex that is not a node),
 * STBEM_ERR_CUDA. */
int stbem_domain_create(stbem_ctx* ctx, const stbem_mesh* mesh, const double* host_nodes, int n_nodes,
                        const int* host_tris, int n_tris, stbem_domain** out);
void stbem_domain_destroy(stbem_domain* dom);
/* Sizes, the number of triangle colours (one assembly launch each) and, if
 * host_bnode is not NULL, the node index of every boundary vertex (n_x ints). */
int stbem_domain_info(const stbem_domain* dom, int* n_nodes, int* n_tris, int* n_colors, int* host_bnode);
/* n_t * n_x * n_nodes * sizeof(double). */
int stbem_m0_bytes(const stbem_domain* dom, size_t* bytes);
/* dev_M0[m][i][j] (FP64, stbem_m0_bytes, caller-owned): overwritten.
 * Deterministic (fixed summation order).  Errors: STBEM_ERR_ARG,
 * STBEM_ERR_CUDA. */
int stbem_m0_assemble(stbem_ctx* ctx, const stbem_domain* dom, double* dev_M0);
/* Matrix-free product: dev_y[b][m][i] += scale * (M_h^0 dev_u0[b])[m][i] for
 * b < n_rhs, dev_u0[b] the n_nodes nodal values, computed with the same rule
 * as stbem_m0_assemble without storing M_h^0.  n_t <= 6144, n_x <= 65535.  Workspace:
 * stbem_m0_apply_workspace_bytes (per-block partial sums).  Errors:
 * STBEM_ERR_ARG, STBEM_ERR_NOMEM (workspace too small), STBEM_ERR_CUDA. */
int stbem_m0_apply_workspace_bytes(const stbem_domain* dom, size_t* bytes);
int stbem_m0_apply(stbem_ctx* ctx, const stbem_domain* dom, int n_rhs, const double* dev_u0, double scale,
                   double* dev_y, void* dev_work, size_t work_bytes);
/* Evaluation of u in Q by the representation formula (Section 1, eq. (2)):
 *   u_h(x, t) = int_Omega U*(x - y, t) u0_h(y) dy + 1/alpha int_Sigma U* w_h
 *             - 1/alpha int_Sigma d_{n_y} U* g_h
 * at n_points points dev_xy[2p], [2p+1] and times dev_t[p] (device arrays),
 * with w_h = dev_w[n][i] (piecewise constant, e.g. the solution of
 * stbem_solve), g_h = dev_g[n][p] (vertex values per step, as stbem_rhs and
 * stbem_planewave_data produce) and u0_h = dev_u0[j] on dom's nodes (dom and
 * dev_u0 NULL: u_0 = 0).  Time integrals exact; space by the repository's
 * rule: 16 / 12 / 8 Gauss points per segment at distance below 2 h / 4 h /
 * beyond, and per triangle the collapsed rule with the order of the M_h^0
 * step table at rho^2 = 4 t / (alpha diam^2).  Meant for points inside the
 * domain at least half a segment from the boundary, 0 < t <= T (no check of
 * the points; the times are not checked against T).  dev_u: n_points values.
 * Errors: STBEM_ERR_ARG (NULL arrays, u0 without a domain, a domain of
 * another mesh), STBEM_ERR_CUDA. */
int stbem_evaluate(stbem_ctx* ctx, const stbem_mesh* mesh, const stbem_domain* dom, int n_points,
                   const double* dev_xy, const double* dev_t, const double* dev_w, const double* dev_g,
                   const double* dev_u0, double* dev_u);
/* Data of the Section 4 example u(x, t) = exp(-t/alpha) sin(x . d),
 * d = (cos theta, sin theta) (the paper: theta = pi/8): dev_g[n][p] the time
 * average of u at vertex p over tau_n, dev_u0[j] = u(y_j, 0) at the nodes.
 * Either pointer may be NULL.  Errors: STBEM_ERR_ARG, STBEM_ERR_CUDA. */
int stbem_planewave_data(stbem_ctx* ctx, const stbem_domain* dom, double theta, double* dev_g, double* dev_u0);

#ifdef __cplusplus
}
#endif
#endif /* STBEM_H */
