/*
 * ssv.h -- C ABI of the GB300 shifted-system solver.
 *
 * Solves (A - sigma_j I) X_j = B for many complex shifts sigma_j and m
 * right-hand sides, the problem of Bosner, Bujanovic and Drmac, "Parallel
 * solver for shifted systems in a hybrid CPU-GPU framework" (Sec. 1), by
 *   (1) one reduction of (A, B, C) to controller-Hessenberg form
 *       (Algorithm 1, Sec. 2): H = Q^T A Q upper m-Hessenberg
 *       (H(i,j) = 0 for i > j + m), R = Q^T B upper triangular, Ct = C Q;
 *   (2) for every shift, the blocked elimination of the m subdiagonals of
 *       H - sigma I from the bottom up with a sliding window of n_b + m
 *       columns (Sec. 3.1, Algorithm 8), back substitution against R(1:m,1:m),
 *       and optionally G = Ct Xhat.
 *
 * Conventions
 *   - All matrices are column-major.  Leading dimensions are in elements.
 *   - Complex arrays are interleaved (re, im) doubles, the layout of
 *     complex128 / cuDoubleComplex; their leading dimension counts complex
 *     elements.
 *   - Every pointer named "device" must point to memory of the current CUDA
 *     device; "host" pointers to host memory.  All work is enqueued on the
 *     given stream (a cudaStream_t passed as void*, NULL = legacy default
 *     stream) and is stream-ordered: inputs must stay valid until the stream
 *     passes the call, outputs are valid once it does.
 *   - Return value 0 = success, negative = failure (SSV_E*); no call throws,
 *     traps or aborts.  ssv_strerror() names a code.  After SSV_ECUDA the
 *     CUDA error is also retrievable with ssv_last_cuda_error().
 *   - Per-shift outcomes are reported in a device int array (SSV_SHIFT_*).
 */
#ifndef SSV_H
#define SSV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define SSV_OK 0
#define SSV_EINVAL (-1)   /* bad argument (size, pointer, leading dimension, option) */
#define SSV_ENOMEM (-2)   /* device allocation failed */
#define SSV_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define SSV_ETIMEOUT (-4) /* a bounded device wait gave up */
#define SSV_ENOTSUP (-5)  /* option combination not supported */
#define SSV_ESCRATCH (-6) /* problem too large for ssv_solve_noalloc's fixed scratch */

/* ---- per-shift status (device int array, one entry per shift) --------- */
#define SSV_SHIFT_OK 0
#define SSV_SHIFT_SINGULAR 1      /* singular to working precision: a diagonal entry of the
                                     triangular factor has modulus <= n eps ||H - sigma I||_F */
#define SSV_SHIFT_NOT_CONVERGED 2 /* refinement stopped above the tolerance */
#define SSV_SHIFT_NONFINITE 3     /* a NaN / Inf appeared */

/* ---- options ----------------------------------------------------------- */
#define SSV_FP64 0  /* every step in double / complex128 */
#define SSV_MIXED 1 /* a first solve of about 48 bits (by default the SSV_SPLIT
                       sweep with its tensor-core trailing update, else
                       double-float; see ssv_opts.first), certified per shift by
                       an FP64-accurate residual (tensor cores for m <= 16),
                       complex64 correction sweeps, FP64 re-solve of shifts that
                       miss the tolerance */
#define SSV_DFLOAT 2 /* the window panels (reflectors formed in double-word
                        scalars) and the bulk updates of the rows above each
                        block (the Z1 P1 and Z2 P2 products, most of the work) in
                        double-float arithmetic on the FP32 pipe: pairs of FP32
                        words, exact FMA products, two-sum accumulation (about 48
                        significant bits; no refinement).  A shift is reported
                        singular when a finalised diagonal entry is <= n 2^-47
                        ||H - sigma I||_F.  Entries of H - sigma I and their
                        squares must be within the FP32 exponent range (moduli
                        between about 1e-18 and 1e18).  ssv_solve, the
                        many-systems launch and batch plans. */

#define SSV_SPLIT 3 /* the sweep as phases over all shifts per block step, with
                       the trailing update Z1 P1 (the product with the shared
                       columns of H, most of the work) on the tensor cores as
                       error-free BF16 digit products (H and the block transforms
                       split into seven 7-bit digits, exact FP32 accumulation per
                       level, about 48 significant bits) and the panels and Z2 P2
                       in double-float as in SSV_DFLOAT; no refinement.
                       m <= 16, n > m, n_b = 128, Householder panel; ssv_solve and
                       ssv_tf_norm2 (ssv_solve_many solves the systems one after
                       another).  Singularity threshold as SSV_DFLOAT. */

#define SSV_G 0    /* out(p x m) = C X = Ct Xhat                             */
#define SSV_TF 1   /* out(p x m) = C (sigma I - A)^{-1} B = -Ct Xhat (Sec. 2) */
#define SSV_XHAT 2 /* out(n x m) = Xhat = (H - sigma I)^{-1} R                */
#define SSV_X 3    /* out(n x m) = X = Q Xhat = (A - sigma I)^{-1} B          */

/* first solve of the mixed path (ssv_opts.first) */
#define SSV_FIRST_DFLOAT 0 /* double-float sweep (about 48 bits): refinement usually
                              only certifies it */
#define SSV_FIRST_TENSOR 2 /* the SSV_SPLIT sweep (tensor-core trailing update, about
                              48 bits; default); where SSV_SPLIT does not apply
                              (m > 16 or n <= m) the double-float sweep is used */
#define SSV_FIRST_C64 1    /* complex64 sweep (the correction sweep started from
                              Xhat = 0): refinement has to win back every digit
                              beyond single precision, and shifts whose condition
                              number times 2^-24 is not well below 1 stagnate and
                              go to the FP64 re-solve */

/* panel factorisation of each window block (FP64 sweeps) */
#define SSV_PANEL_HOUSEHOLDER 0 /* one complex reflector per row (default) */
#define SSV_PANEL_GIVENS 1      /* Givens rotations in the greedy parallel order of
                                   Algorithm 9 (Sec. 3.2); n_b <= 32, m <= 32 */

typedef struct ssv_opts {
  int precision;           /* SSV_FP64, SSV_MIXED, SSV_DFLOAT or SSV_SPLIT */
  int mode;                /* SSV_G, SSV_TF, SSV_XHAT, SSV_X */
  int nb;                  /* rows per elimination block n_b; 0 = default */
  int max_refine;          /* SSV_MIXED: maximum refinement sweeps */
  double tol;              /* SSV_MIXED: target normwise backward error */
  int panel;               /* SSV_PANEL_HOUSEHOLDER or SSV_PANEL_GIVENS (ssv_solve, FP64) */
  int first;               /* SSV_MIXED: SSV_FIRST_DFLOAT, SSV_FIRST_C64 or SSV_FIRST_TENSOR */
} ssv_opts;

typedef struct ssv_handle_s* ssv_handle;

/* Fill *o with the defaults: FP64, SSV_G, nb = 0, max_refine = 8,
 * tol = 1e-13, panel = SSV_PANEL_HOUSEHOLDER, first = SSV_FIRST_TENSOR.  (The mixed path certifies each
 * shift with a residual whose own error, as a backward error, is below 5e-15
 * for m <= 16 (the tensor-core residual) and about 1e-14 for wider m (the
 * double-float residual); 1e-13 stays above both.) */
void ssv_default_opts(ssv_opts* o);

/*
 * ssv_reduce -- controller-Hessenberg reduction (Algorithm 1, Sec. 2).
 *   n >= 1, 1 <= m <= n, p >= 0.
 *   A (device) n x n double, lda >= n;  B (device) n x m double, ldb >= n;
 *   C (device) p x n double, ldc >= max(1, p) (may be NULL when p == 0).
 * A, B and C are read only.  On success *out receives a handle that owns
 * device copies of H (n x n), R (n x m), Ct (p x n) and the Householder
 * vectors of Q, all FP64.  The reduction runs entirely on the GPU in FP64, as
 * one persistent cooperative kernel whose phases are separated by a bounded
 * grid barrier; the call returns after it has completed on `stream`.
 * Errors: SSV_EINVAL (sizes / pointers), SSV_ENOMEM, SSV_ECUDA, SSV_ETIMEOUT
 * (a barrier wait ran out; no result); *out is then left NULL.
 */
int ssv_reduce(int n, int m, int p, const double* A, long long lda, const double* B,
               long long ldb, const double* C, long long ldc, void* stream, ssv_handle* out);

/* arithmetic of the reduction's bulk products (ssv_reduce_arith) */
#define SSV_REDUCE_FP64 0   /* every product on the FP64 pipe (ssv_reduce) */
#define SSV_REDUCE_TENSOR 1 /* two levels of blocking (Sec. 2.1: blocks of b = floor(128/m) m
                               columns split into mini-blocks of m), the products A V_s,
                               V^T A and the block's rank-b updates as error-free BF16 digit
                               products on the tensor cores (eight 7-bit digits per value,
                               levels accumulated exactly in FP32, FP64 result, about the
                               accuracy of an FP64 product); panels, T and the small
                               products in FP64.  m <= 64, n >= 2 */

/*
 * ssv_reduce_arith -- ssv_reduce with the arithmetic of its bulk products
 * chosen by `arith` (SSV_REDUCE_FP64 or SSV_REDUCE_TENSOR).  Same arguments,
 * ownership, result layout (H with the Householder vectors of Q_A below the
 * m-th subdiagonal, R with those of Q_B below its diagonal, tau of every
 * reflector) and errors as ssv_reduce; SSV_ENOTSUP when SSV_REDUCE_TENSOR
 * is asked for m > 64, n < 2, or an n so large that a panel slice exceeds a
 * CTA's shared memory (about 77000 rows at m = 16).  The scratch of the
 * tensor-core form is about (p + n) n x 47 bytes (1.17 GB at n = 5000), taken from the library's
 * memory pool for the duration of the call.
 */
int ssv_reduce_arith(int n, int m, int p, const double* A, long long lda, const double* B,
                     long long ldb, const double* C, long long ldc, int arith, void* stream,
                     ssv_handle* out);

/*
 * ssv_solve -- the batched shifted m-Hessenberg solve (Sec. 3, Algorithm 8).
 *   s >= 0 shifts, shifts (device) = s interleaved complex doubles.
 *   o: options (NULL = defaults).
 *   out (device, complex): for SSV_G / SSV_TF a p x (s*m) matrix with
 *     ldo >= max(1, p); block j (columns j*m .. j*m+m-1) is G(sigma_j)
 *     (the layout of Algorithm 8's output).  For SSV_XHAT / SSV_X an
 *     n x (s*m) matrix with ldo >= n.
 *   status (device, may be NULL): s ints, SSV_SHIFT_*.
 *   resid (device, may be NULL): s doubles, the normwise backward error
 *     ||(H - sigma I) Xhat - R||_F / (||H - sigma I||_F ||Xhat||_F + ||R||_F)
 *     of each shift's computed Xhat.
 * The handle is read only; concurrent calls on one handle from different
 * streams are safe (each call allocates its own stream-ordered scratch).
 * Errors: SSV_EINVAL, SSV_ENOTSUP, SSV_ENOMEM, SSV_ECUDA.
 */
int ssv_solve(ssv_handle h, int s, const double* shifts, const ssv_opts* o, double* out,
              long long ldo, int* status, double* resid, void* stream);

/*
 * ssv_solve_rhs -- one right-hand side per shift (Sec. 3.3, the systems
 * (A - sigma_l I) x_l = B bhat_l that interpolatory model reduction needs):
 * the same sweep as ssv_solve, whose final m x m step solves for the single
 * column R(1:m, 1:m) bhat_l (the reduced right-hand side has at most m
 * nonzero entries) instead of the m columns of R.
 *   bhat (device): complex m x s, column l = bhat_l, ld ldb >= m.
 *   o: precision SSV_FP64 only (SSV_MIXED -> SSV_ENOTSUP); mode
 *     SSV_X     out column l = x_l = (A - sigma_l I)^{-1} B bhat_l (n rows),
 *     SSV_XHAT  out column l = Q^T x_l (reduced coordinates, n rows),
 *     SSV_G     out column l = C x_l = G(sigma_l) bhat_l (p rows),
 *     SSV_TF    out column l = -C x_l = C (sigma_l I - A)^{-1} B bhat_l.
 *   out (device): complex, (n or p) x s, ld ldo >= n (or max(1, p)).
 *   status (device, may be NULL): s ints, SSV_SHIFT_*.
 * Errors: SSV_EINVAL, SSV_ENOTSUP, SSV_ENOMEM, SSV_ECUDA.
 */
int ssv_solve_rhs(ssv_handle h, int s, const double* shifts, const double* bhat, long long ldb,
                  const ssv_opts* o, double* out, long long ldo, int* status, void* stream);

/*
 * ssv_solve_trans -- the transposed systems (A - sigma_l I)^T x_l = C^T chat_l
 * (Sec. 3.3; plain transpose, not conjugate), one right-hand side per shift.
 * In reduced coordinates (H - sigma I)^T xt = C~^T chat with x = Q xt.  With J
 * the reversal permutation, J (H - sigma I)^T J is upper m-Hessenberg again,
 * so the bottom-up sweep of ssv_solve solves it for the dense right-hand side
 * J C~^T chat, back-substituting against each finalised column as it appears.
 *   chat (device): complex p x s, column l = chat_l, ld ldc >= max(1, p);
 *     the handle must have p >= 1.
 *   o: precision SSV_FP64 only; mode SSV_X (out column l = x_l) or SSV_XHAT
 *     (out column l = Q^T x_l); other modes -> SSV_ENOTSUP.
 *   out (device): complex n x s, ld ldo >= n.
 *   status (device, may be NULL): s ints, SSV_SHIFT_*.
 * Each call allocates (stream-ordered) an n x n flipped copy of H, n x s
 * right-hand sides and the per-block window state; the handle is not changed.
 * Errors: SSV_EINVAL, SSV_ENOTSUP, SSV_ENOMEM, SSV_ECUDA.
 */
int ssv_solve_trans(ssv_handle h, int s, const double* shifts, const double* chat, long long ldc,
                    const ssv_opts* o, double* out, long long ldo, int* status, void* stream);

/*
 * ssv_givens_schedule -- the greedy parallel annihilation schedule that
 * SSV_PANEL_GIVENS uses (Algorithm 9, Sec. 3.2), for a window block of `rows`
 * rows and rows + m columns.  Host-only (no device work).
 *   rot (host, capacity max_rot): triples r, c1, c2 (1-based, as in the
 *     paper's worked example): the zero at (r, c1) is introduced with (r, c2);
 *   off (host, capacity max_steps + 1): step t holds rotations off[t] ..
 *     off[t+1]-1;  *nsteps: the number of steps.
 * Returns the number of rotations (rows * m), or SSV_EINVAL (bad sizes,
 * NULL pointers, or capacities too small).
 */
int ssv_givens_schedule(int rows, int m, int* rot, int max_rot, int* off, int max_steps,
                        int* nsteps);

/*
 * ssv_tf_norm2 -- ||C (sigma_j I - A)^{-1} B||_2 for every shift: the function
 * whose level sets {z : ||C (zI - A)^{-1} B||_2 >= 1/eps} are the structured
 * pseudospectra of (A, B, C) (Sec. 1).  Solves for G(sigma_j) with the
 * precision of o (mode ignored), then the largest singular value of each
 * p x m block by Jacobi on G^H G or G G^H (one warp per shift).
 *   norms (device): s doubles (NaN for a shift whose G is not finite);
 *   status (device, may be NULL): s ints from the solve.
 *   Requires 1 <= min(m, p) <= 32.
 * Errors: SSV_EINVAL, SSV_ENOTSUP, SSV_ENOMEM, SSV_ECUDA.
 */
int ssv_tf_norm2(ssv_handle h, int s, const double* shifts, const ssv_opts* o, double* norms,
                 int* status, void* stream);

/* residual methods of ssv_backward_error */
#define SSV_RESID_FP64 0   /* FP64 products on the FP64 pipe */
#define SSV_RESID_TENSOR 1 /* error-free BF16 digit splitting of H and Xhat (Ozaki
                              scheme, 7-bit digits, 36 slice products accumulated
                              exactly in FP32 on the tensor cores, combined in
                              double-float): about 2^-50 of ||H|| ||Xhat||; m <= 16 */

/*
 * ssv_backward_error -- normwise backward error of caller-supplied solutions
 * Xhat of (H - sigma_j I) Xhat = R (reduced coordinates, Sec. 2):
 *   eta_j = ||(H - sigma_j I) Xhat_j - R||_F / (||H - sigma_j I||_F ||Xhat_j||_F + ||R||_F),
 * the certificate that the mixed path's refinement tests against its tolerance.
 *   xhat (device): complex128, shift j at xhat + 2 j m ldx doubles, n x m,
 *     leading dimension ldx >= n (the SSV_XHAT output layout);
 *   method: SSV_RESID_FP64 or SSV_RESID_TENSOR;
 *   eta (device): s doubles (NaN when Xhat_j is not finite, or, for
 *     SSV_RESID_TENSOR, when a bounded wait for the tensor cores gave up).
 * Stream-ordered; scratch is allocated and freed on `stream`.
 * Errors: SSV_EINVAL, SSV_ENOTSUP (SSV_RESID_TENSOR with m > 16), SSV_ENOMEM,
 * SSV_ECUDA.
 */
int ssv_backward_error(ssv_handle h, int s, const double* shifts, const double* xhat,
                       long long ldx, int method, double* eta, void* stream);

/*
 * ssv_solve_many -- many reduced systems of uneven n, m and shift counts in
 * one persistent launch (FP64 and SSV_DFLOAT: one kernel over a cost-ordered
 * worklist of (system, shift) items, Sec. 3 applied to several systems at
 * once; MIXED: the systems are solved one after another on the stream).
 *   nsys systems; hs[k] handle, s[k] shifts at shifts[k] (device), results in
 *   outs[k] (device, layout as ssv_solve with leading dimension ldos[k]),
 *   statuses in status[k] (device, or status == NULL / status[k] == NULL).
 *   hs, s, shifts, outs, ldos, status are host arrays.  Modes SSV_G, SSV_TF,
 *   SSV_XHAT.  All handles must belong to the current device.
 * Stream-ordered like ssv_solve: the per-call plan (descriptors, worklist,
 * scratch) is allocated and freed on `stream` (on the legacy default stream,
 * NULL, the call synchronises that stream before returning).
 * Errors: SSV_EINVAL, SSV_ENOTSUP, SSV_ENOMEM, SSV_ECUDA.
 */
int ssv_solve_many(int nsys, const ssv_handle* hs, const int* s, const double* const* shifts,
                   const ssv_opts* o, double* const* outs, const long long* ldos,
                   int* const* status, void* stream);

/*
 * Batch plans: the FP64 multi-system solve with everything fixed up front, so
 * that ssv_batch_run is a single kernel launch with constant arguments that
 * can be captured into a CUDA graph and replayed; between runs the caller may
 * rewrite the contents (not the addresses) of the shift buffers.
 *   ssv_batch_create: arguments as ssv_solve_many (precision SSV_FP64 or SSV_DFLOAT;
 *   nb = 0 takes the autotuned or default block width per system); allocates
 *   the plan (device descriptors, worklist, scratch) synchronously.
 *   ssv_batch_run: enqueue the batch on `stream`.
 *   ssv_batch_destroy: free the plan (after synchronising the device).
 */
typedef struct ssv_batch_s* ssv_batch;
int ssv_batch_create(int nsys, const ssv_handle* hs, const int* s, const double* const* shifts,
                     const ssv_opts* o, double* const* outs, const long long* ldos,
                     int* const* status, ssv_batch* out);
int ssv_batch_run(ssv_batch b, void* stream);
void ssv_batch_destroy(ssv_batch b);

/*
 * ssv_autotune -- choose the elimination block width n_b for this handle,
 * precision and mode by timing each candidate (FP64: 32, 48, 64, 96, 128;
 * MIXED: 16, 24, 32, 48, 64) on the
 * given s shifts (device) with CUDA events; writes the results to out
 * (scratch for the caller, layout as ssv_solve).  The choice is cached for
 * the process and used by every later call with o->nb == 0 on a system of the
 * same (n, m, p).  Synchronises `stream`.  *best_nb receives the choice and
 * *best_ms (may be NULL) its time.
 */
int ssv_autotune(ssv_handle h, int s, const double* shifts, const ssv_opts* o, double* out,
                 long long ldo, void* stream, int* best_nb, float* best_ms);

/*
 * ssv_solve_noalloc -- ssv_solve without any device allocation.  The paper has
 * no counterpart; this entry point exists for callers that cannot allocate
 * device memory when they solve (an external allocator or framework owns all
 * device memory during their step, a device-memory budget fixed in advance,
 * or a latency-critical loop where an allocation may not stall or fail).
 *
 *   Same arguments and results as ssv_solve with precision SSV_FP64, the
 *   Householder panel and mode SSV_G, SSV_TF or SSV_XHAT (the same n_b as
 *   ssv_solve, an autotuned one included, so the results agree); there is no
 *   resid output.  The handle, shifts, out and status are the caller's,
 *   allocated beforehand.
 *   Scratch: a fixed 64 MiB array inside the library.  It is part of the
 *   module that holds the FP64 solve kernels, so it is reserved on every GPU
 *   where any FP64 or double-float solve (not only this entry point) has run,
 *   until the process exits.  One shift's window needs 16 * (p + n) * m bytes
 *   (plus 16 * n * m for SSV_XHAT); sizes where that exceeds 64 MiB return
 *   SSV_ESCRATCH, and smaller sizes run with as many thread blocks as fit
 *   (fewer than ssv_solve uses when n * m is large; each then solves more
 *   shifts in turn).
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) and caches it; under lazy module loading that
 *   lookup may load the module, which allocates device memory.  Make the
 *   first call outside any region where allocation is forbidden, and before
 *   any stream capture.
 *   Every call uses the same array and leaves its contents behind: calls
 *   whose executions overlap on the GPU (different streams, or different host
 *   threads) race on it and give wrong results; serialize them.
 * Errors: SSV_EINVAL, SSV_ENOTSUP (precision, mode, panel other than
 * SSV_PANEL_HOUSEHOLDER, m > 32), SSV_ESCRATCH, SSV_ECUDA.
 */
int ssv_solve_noalloc(ssv_handle h, int s, const double* shifts, const ssv_opts* o, double* out,
                      long long ldo, int* status, void* stream);

/*
 * ssv_apply_q -- X = Q Xhat (Sec. 2: X = Q Xhat in original coordinates).
 *   Xhat (device, complex) n x ncols, ldx >= n; X (device, complex) n x ncols,
 *   ldX >= n.  X may equal Xhat (in place).
 */
int ssv_apply_q(ssv_handle h, int ncols, const double* Xhat, long long ldx, double* X,
                long long ldX, void* stream);

/*
 * ssv_get_reduced -- copy the reduced triple out of the handle (device
 * destinations, FP64, column-major; entries of H below the m-th subdiagonal
 * and of R below the diagonal are written as exact zeros).  Any destination
 * may be NULL to skip it.  H: n x n (ldh >= n); R: n x m (ldr >= n);
 * Ct: p x n (ldc >= max(1, p)).
 */
int ssv_get_reduced(ssv_handle h, double* H, long long ldh, double* R, long long ldr, double* Ct,
                    long long ldc, void* stream);

/*
 * ssv_load_reduced -- build a handle from a stored reduced triple (restoring
 * a checkpoint written with ssv_get_reduced, or a system already in
 * controller-Hessenberg form).  H (device) n x n, ldh >= n, read only on and
 * above the m-th subdiagonal; R (device) n x m, ldr >= n, read only on and
 * above the diagonal; Ct (device) p x n, ldc >= max(1, p).  The handle has no
 * Q: ssv_apply_q and SSV_X return SSV_ENOTSUP on it.  Errors as ssv_reduce.
 */
int ssv_load_reduced(int n, int m, int p, const double* H, long long ldh, const double* R,
                     long long ldr, const double* Ct, long long ldc, void* stream,
                     ssv_handle* out);

/* Dimensions of a handle.  Any output pointer may be NULL. */
int ssv_dims(ssv_handle h, int* n, int* m, int* p);

/*
 * ssv_footprint -- device bytes one ssv_solve call with these sizes and
 * options allocates for scratch (in addition to the handle), for admission
 * control.  *bytes receives the count.
 */
int ssv_footprint(int n, int m, int p, int s, const ssv_opts* o, size_t* bytes);

/* Bytes the handle of an (n, m, p) system keeps on the device. */
int ssv_handle_bytes(int n, int m, int p, size_t* bytes);

/* Release a handle (stream-ordered on the stream given to ssv_reduce after a
 * device synchronisation of that stream).  NULL is ignored. */
void ssv_destroy(ssv_handle h);

/* Static string naming a return code. */
const char* ssv_strerror(int code);

/* Scratch memory.  Every call that allocates scratch (all but
 * ssv_solve_noalloc) takes it stream-ordered from a memory pool the library
 * keeps per device; freed scratch stays mapped in the pool for the next call
 * (so repeated solves do not map their scratch anew after each
 * synchronisation), up to the largest amount used at once.  ssv_pool_trim
 * returns the current device's pool memory beyond keep_bytes to the system
 * (memory of calls still in flight is kept).  Errors: SSV_ECUDA. */
int ssv_pool_trim(size_t keep_bytes);

/* The last CUDA error code seen by this thread's calls (0 if none). */
int ssv_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads); differences of two reads count the launches of the calls between
 * them.  Measurement aid; the paper has no counterpart. */
long long ssv_kernel_launches(void);

/* Refinement counters of the mixed path (measurement aid; the paper has no
 * counterpart), kept on the current device and accumulated over every
 * SSV_MIXED solve on it:
 *   *corrections: shift-sweeps of correction (shifts active in a correction
 *     sweep, summed over the sweeps; with SSV_FIRST_C64 the first solve is not
 *     counted);
 *   *resolves: shifts re-solved by the FP64 sweep after refinement missed the
 *     tolerance, stagnated or met a singular first solve.
 * Either pointer may be NULL.  reset != 0 clears the counters after reading.
 * Synchronises the device.  Errors: SSV_ECUDA. */
int ssv_refine_counts(long long* corrections, long long* resolves, int reset);

/* Phase tracer (measurement aid; the paper has no counterpart).  When
 * enabled, the library records CUDA events on the launching stream around its
 * internal phases ("reduce", "solve_fp64", "mixed_sweep0", "mixed_residual",
 * "mixed_correction", "mixed_fallback", "batch").  ssv_trace_read
 * synchronises the recorded events and returns up to `max` phases: names
 * (NUL-terminated, `name_len` bytes each), total milliseconds and call
 * counts; *count receives the number of distinct phases.  Keep the tracer off
 * while a stream is captured into a CUDA graph. */
int ssv_trace_enable(int on);
int ssv_trace_reset(void);
int ssv_trace_read(int max, char* names, int name_len, float* total_ms, int* calls, int* count);

/* Self-test of the bounded grid barrier used by ssv_reduce (the paper has no
 * counterpart): launches a small cooperative kernel in which one block never
 * arrives, so the others give up after `spin_limit` short naps.  Returns
 * SSV_ETIMEOUT when the timeout path works (the device stays usable), SSV_OK
 * if it did not trigger, SSV_EINVAL / SSV_ECUDA on errors.  Synchronises. */
int ssv_selftest_barrier(long long spin_limit, void* stream);

/* Arithmetic peak probe (measurement aid; the paper has no counterpart):
 * runs independent fused multiply-add chains on every SM of the current
 * device for a few milliseconds, synchronises `stream`, and stores the best
 * of three runs in *tflops.  kind 0 = FP64 (DFMA), 1 = FP32 (FFMA).
 * Errors: SSV_EINVAL, SSV_ENOMEM, SSV_ECUDA. */
int ssv_peak_probe(int kind, void* stream, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* SSV_H */
