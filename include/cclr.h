/*
 * libcclr: relativistic CCSD linear response on one NVIDIA B300 (sm_103a).
 *
 * The library implements the hot path of arXiv 2307.14296 (Yuan, Halbert, Pototschnig, Papadopoulos,
 * Coriani, Visscher, Pereira Gomes, "Formulation and implementation of frequency-dependent linear
 * response properties with relativistic coupled cluster theory for GPU-accelerated computer
 * architectures"): the CCSD Jacobian-times-vector products (sigma vectors) over complex,
 * antisymmetrized spinor integrals, the damped first-order response solve
 *     (A - (w + i gamma)) t^X = -xi^X                   (Sec. 2.4, Eq. LR response equation_cpp)
 * the Lambda (left) solve  t-bar A = -eta             (Sec. 2.3), and the symmetric CC-CC response
 * function <<X;Y>>_w                                    (Sec. 2.3, Eq. CC-CC response function).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are interleaved (re, im) doubles: cclr_c128.
 *  - n_occ = o, n_vir = v; spinors 0..o-1 are occupied, o..o+v-1 virtual.
 *  - A pair index over p<q inside one index range is P(p,q) = q*(q-1)/2 + p.
 *  - Excitation vectors ("amplitude layout") hold unique elements only:
 *        [ singles t_i^a at i*v + a  (o*v entries) | doubles t_ij^ab at P(i,j)*Pv + P(a,b) ]
 *    with Pv = v(v-1)/2, Po = o(o-1)/2; length N = o*v + Po*Pv.  Sums over this layout count
 *    each unique doubles element once.  Response-function contractions are bilinear (no
 *    conjugation); the Hermitian product b^H c is used only inside the iterative solver.
 *  - Unless a call says otherwise, pointers are HOST pointers; the caller keeps ownership and the
 *    library copies what it needs.  Calls are synchronous with respect to the host.
 *  - No call throws.  Every failure returns a status other than CCLR_OK and sets a message that
 *    cclr_last_error() returns until the next call on the same context.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef CCLR_H
#define CCLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cclr_ctx cclr_ctx;
typedef struct { double re, im; } cclr_c128;

typedef enum {
  CCLR_OK = 0,
  CCLR_E_ARG = 1,      /* invalid argument (size, pointer, option) */
  CCLR_E_NOCONV = 2,   /* iteration limit reached; the best iterate is kept and readable */
  CCLR_E_OOM = 3,      /* device allocation failed */
  CCLR_E_CUDA = 4,     /* a CUDA runtime call failed (message carries cudaGetErrorString) */
  CCLR_E_STATE = 5,    /* call-order violation (e.g. cc_lambda before cc_ground) */
  CCLR_E_TIMEOUT = 6   /* a device-side bounded wait expired */
} cclr_status;

/* Arithmetic used for the large contractions (the paper computes in complex FP64, Sec. 2.4).
 *  CCLR_FP64      complex FP64 everywhere (DFMA on the CUDA cores).
 *  CCLR_TC_BF16X3 the ladder and ring contractions (and every other large K-major GEMM) run on
 *                 the tensor cores from split-BF16 operands x = x0 + x1 (products x0y0 + x0y1 +
 *                 x1y0, FP32 accumulation; ~1e-5 relative per contraction).
 *  CCLR_TC_BF16X6 as above with three slices and six products: the FP32-class tensor-core mode
 *                 (FP32 complex accuracy, ~1e-6 relative per contraction, limited by the FP32
 *                 accumulation over long K).
 *  CCLR_TC_F64    FP64-class tensor-core mode: every operand row is cut into five fixed-point
 *                 BF16 digits on a per-row exponent grid (Ozaki splitting), the 15 digit products
 *                 above 2^-40 are summed on the tensor cores, the two leading digit groups exactly
 *                 in 256-deep chunks, and the chunk sums in float-float; ~1e-11 relative to the
 *                 product of the row maxima.  Operand magnitudes must lie within the binary32
 *                 range.  The solvers treat this mode like CCLR_FP64 (FP64 vector arithmetic, no
 *                 convergence floors).
 *  In the BF16X3/BF16X6 modes the solvers' vector passes run in FP32 arithmetic and the iterations
 *  stop at floors relative to the right-hand side (see cclr_options.refine); small solves and the
 *  response-function contraction stay in FP64 in every mode. */
typedef enum {
  CCLR_FP64 = 0,
  CCLR_TC_BF16X3 = 2,
  CCLR_TC_BF16X6 = 3,
  CCLR_TC_F64 = 4,
  CCLR_BF16X2_TC = CCLR_TC_BF16X3, /* other names: split BF16 (two slices per operand) */
  CCLR_FP32_TC = CCLR_TC_BF16X6    /*              the FP32-class tensor-core mode */
} cclr_precision;

typedef struct {
  double tol;          /* residual 2-norm target of the response solves (default 1e-8)        */
  double ground_tol;   /* residual 2-norm target of the CCSD and Lambda equations (1e-10)      */
  int maxit;           /* iteration limit of every iterative solve (default 100)               */
  int max_subspace;    /* Davidson trial-space limit per right-hand side (default 96)          */
  int precision;       /* a cclr_precision value (default CCLR_FP64)                           */
  int batch;           /* right-hand sides per batched sigma launch, 0 = automatic             */
  /* FP64 iterative refinement in the CCLR_TC_BF16X3 / CCLR_TC_BF16X6 modes (default 1).  With
   * refine = 1, the Hbar intermediates, xi, eta and the Hessian products are formed in the
   * FP64-class mode (CCLR_TC_F64), and every iterative solve (CCSD, Lambda, response) first runs
   * in the mixed mode until its residual reaches refine_tol times the norm of its right-hand side
   * (CCSD: of its first residual), then continues from the compressed solutions with FP64-class
   * sigma products and FP64 residuals, norms and orthogonalisation until tol / ground_tol is met.
   * CCLR_E_NOCONV is returned if it is not met within maxit.  With refine = 0 the mixed solve
   * stops at that floor (or when it stagnates within 5x of it) and returns CCLR_OK; the residual
   * reached is in cclr_stats.max_residual. */
  int refine;
  double refine_tol;   /* mixed-phase floor relative to the right-hand side, 0 = 2e-5         */
  /* Tile autotuning of the split-BF16 GEMM kernel (default 1): the first two launches of every
   * GEMM shape try a 128-row and a 64-row tile (timed with CUDA events on the context's stream),
   * later launches use the faster.  With the environment variable CCLR_AUTOTUNE_CACHE naming a
   * file, decisions are read from it at first use and appended to it.  0: 128-row tiles. */
  int autotune;
} cclr_options;

/* Fill *opt with the defaults listed above. */
void cclr_default_options(cclr_options *opt);

/* Create a context on CUDA device `device` (its stream, workspace and all device memory).
 * opt may be NULL (defaults).  Returns CCLR_E_ARG for a bad device, CCLR_E_CUDA otherwise. */
cclr_status cclr_create(cclr_ctx **out, int device, const cclr_options *opt);

/* Free every device allocation of the context.  NULL is ignored. */
void cclr_destroy(cclr_ctx *ctx);

/* Message of the last failed call on this context (empty string if none).  The pointer stays
 * valid until the next call on the context.  ctx may be NULL (returns a static message). */
const char *cclr_last_error(const cclr_ctx *ctx);

/* Load the Hamiltonian (paper Sec. 3 step 1 input: Fock matrix and the six integral classes of
 * Sec. 4, "all six two-electron integral classes").
 *   fock    (o+v)x(o+v) row-major, <p|f|q> at p*(o+v)+q.
 *   blocks  six host arrays, antisymmetrized integrals <pq||rs>, in this order and layout:
 *     [0] oooo <ij||kl>  [P(i,j)][P(k,l)]      [3] ovov <ia||jb>  [i][a][j][b]
 *     [1] ooov <ij||ka>  [P(i,j)][k][a]        [4] ovvv <ia||bc>  [i][a][P(b,c)]
 *     [2] oovv <ij||ab>  [P(i,j)][P(a,b)]      [5] vvvv <ab||cd>  [P(a,b)][P(c,d)]
 *   All other index classes follow from <pq||rs> = -<qp||rs> = -<pq||sr> = conj(<rs||pq>).
 * Requires o >= 2, v >= 2.  Discards any previous ground state, Lambda and response data. */
cclr_status cclr_set_hamiltonian(cclr_ctx *ctx, int n_occ, int n_vir, const cclr_c128 *fock,
                                 const cclr_c128 *const blocks[6]);

/* Solve the ground-state CCSD equations Omega(t) = 0 (paper Sec. 3 step 1) from t = 0 and build
 * the Hbar intermediates of the SI (step 2).  e_corr_out (may be NULL) receives the complex
 * correlation energy, iters_out (may be NULL) the iteration count.  CCLR_E_NOCONV keeps the
 * last amplitudes. */
cclr_status cc_ground(cclr_ctx *ctx, cclr_c128 *e_corr_out, int *iters_out);

/* Solve the Lambda equations t-bar^(0) A = -eta (Sec. 2.3) with left sigma vectors (SI Eqs.
 * sigma_sin-ee-left, sigma_double-ee-left).  Requires cc_ground (else CCLR_E_STATE). */
cclr_status cc_lambda(cclr_ctx *ctx, int *iters_out);

/* Damped linear response (Sec. 2.4 and SI Davidson scheme): for every operator X_k (n_ops
 * Hermitian (o+v)x(o+v) row-major host matrices, contiguous) and every frequency omegas[f] with
 * damping gamma >= 0, solve (A - z) t = -xi^X for the shifts z in {w+ig, -w+ig, w-ig, -w-ig}
 * that the response function needs (duplicates removed).  iters_out (may be NULL) receives
 * n_ops*n_freq iteration counts (max over the shifts of that pair).  The solutions stay in the
 * context.  Requires cc_lambda. */
cclr_status cc_lr_solve(cclr_ctx *ctx, int n_ops, const cclr_c128 *ops, int n_freq,
                        const double *omegas, double gamma, int *iters_out);

/* The symmetric CC-CC response function (Sec. 2.3 Eq. CC-CC response function with the damped
 * frequency of Sec. 2.4): out[f][x][y] = <<X_x;X_y>>_{w_f + i gamma}, out holds
 * n_freq*n_ops*n_ops values.  The polarizability is alpha = -<<mu;mu>>.  Requires cc_lr_solve. */
cclr_status cc_response_function(cclr_ctx *ctx, cclr_c128 *out);

/* Gradient of the CC-CC response function with respect to the property operators, by the adjoint
 * method (Sec. 2.3: the response function is linear in each operator through xi^X and eta^X; the
 * multipliers l of t-bar A-type left equations carry the dependence of t^X on xi^X).  For
 * frequency index f of the last cc_lr_solve and every operator k, four n x n matrices G[k][s],
 * s over the shifts (0: w+ig, 1: -w+ig, 2: w-ig, 3: -w-ig), with
 *   G[k][s] = 1/2 [ eta-density(t^k(w_s)) + xi-density(l) ],  l (A + w_s) = -(eta^k + F t^k(w_s)),
 * where the densities D are the matrices with eta^X . v = sum_pq D_pq X_pq and
 * l . xi^X = sum_pq D_pq X_pq.  For perturbations dX_x and dX_y of operators x and y:
 *   d<<X_x;X_y>>_{w+ig} = sum G[y][0] o dX_x + conj(sum G[y][1] o dX_x)
 *                       + sum G[x][3] o dX_y + conj(sum G[x][2] o dX_y)
 * (o: element-wise product summed over all p, q).  out: n_ops*4*n*n values, [k][s][p][q]
 * row-major.  Costs 4 n_ops left solves and Hessian products; the four left systems of one
 * operator are solved together, each holding 2 max_subspace vectors of N complex values
 * (CCLR_E_OOM if they do not fit).  Requires cc_lr_solve. */
cclr_status cclr_response_gradient(cclr_ctx *ctx, int f, cclr_c128 *out);

/* A synthetic instance generated on the device and installed as the Hamiltonian (as
 * cclr_set_hamiltonian with it), for measurements without host generation and host-to-device
 * copies.  Recipe (the counter-based one of the Python package's synth.counter, bit for bit):
 * Philox4x32-10 (Salmon et al., SC'11), counter (element index lo, hi, stream, 0), key (seed lo,
 * hi); per element a Box-Muller pair from two 53-bit uniforms with logarithm and sine / cosine
 * from fixed-order series in explicitly rounded FP64.  Orbital energies occupied U[-2, -0.5],
 * virtual U[0.3, 4] (stream 0, each range sorted); the six antisymmetrized classes in the packed
 * layouts of cclr_set_hamiltonian with Re, Im ~ N(0, sd^2) per canonical element (streams 1..6;
 * the Hermitian classes real on their diagonal); n_ops Hermitian operators with entries
 * N(0, dip_sd^2) (streams 100 + k) written to ops_out (n_ops x n x n, host or device memory;
 * may be null when n_ops = 0).  Temporary device arrays of the packed class sizes are allocated
 * and freed inside the call.  Errors as cclr_set_hamiltonian; CCLR_E_OOM if the temporaries do not
 * fit. */
cclr_status cclr_set_synthetic(cclr_ctx *ctx, int n_occ, int n_vir, uint64_t seed, double sd, double dip_sd,
                               int n_ops, cclr_c128 *ops_out);

/* eta of the CC energy at the current T: the derivative dE/dt in the amplitude layout (the Lambda
 * equations read t-bar A = -eta; Sec. 2.3 and the SI ground-state Lambda equations).  N values. */
cclr_status cclr_eta_ground(cclr_ctx *ctx, cclr_c128 *out);

/* Left (adjoint) linear systems  l_k (A + w) = -b_k  for nrhs right-hand sides b (nrhs x N, amplitude
 * layout) at the current T, with the shift w = w_re + i w_im (SI left sigma equations
 * sigma_sin-ee-left / sigma_double-ee-left).  b = eta of the energy and w = 0 give Lambda; the
 * response-function gradient uses b = eta^X + F t^X(w).  Solved to cclr_options.tol by the same
 * Davidson and refinement as the Lambda equations; out: nrhs x N.  CCLR_E_NOCONV if the solve
 * does not converge within maxit (out is then not written), CCLR_E_ARG on non-finite input. */
cclr_status cclr_left_solve(cclr_ctx *ctx, int nrhs, const cclr_c128 *rhs, double w_re, double w_im,
                            cclr_c128 *out);

/* The CC-CI response function (Sec. 2.3 Eq. CC-CI response function; EOM-eta of the SI "Linear
 * response" section): the same symmetrization and layout as cc_response_function, from the
 * solutions of the last cc_lr_solve, without the Hessian term.  Requires cc_lr_solve (after
 * cc_lambda); CCLR_E_STATE otherwise. */
cclr_status cc_response_function_ci(cclr_ctx *ctx, cclr_c128 *out);

/* The asymmetric CC-CC response function (Sec. 2.3, the asymmetric form beside Eq. CC-CC
 * response function): with the first-order multipliers of each operator Y,
 *   tbar^Y(z) (A + z) = -(eta^Y + F t^Y(z))   (left sigma products, solved to cclr_options.tol),
 *   f(z) = 1/2 [eta^X t^Y(z) + tbar^Y(z) xi^X],   out[f][x][y] = f(z) + conj(f(-z*)),
 * z = w_f + i gamma, from the solutions t^Y(z), t^Y(-z*) of the last cc_lr_solve.  Same layout
 * as cc_response_function and equal to it for exact solutions (its error is first order in the
 * solution errors, the symmetric form's second order).  Costs 2 n_ops left solves and Hessian
 * products per frequency; the two left systems of one operator and frequency are solved together,
 * each holding 2 max_subspace vectors of N complex values (CCLR_E_OOM if they do not fit).  Requires cc_lr_solve; CCLR_E_STATE otherwise, CCLR_E_NOCONV if a
 * multiplier solve does not converge within maxit (out is then not written). */
cclr_status cc_response_function_asym(cclr_ctx *ctx, cclr_c128 *out);

/* Static-field derivative of the CC-CC response function (Sec. 2.3 Eq. CC-CC response function
 * differentiated): out[f][x][y] = d<<X_x;X_y>>_{w_f + i gamma} / d eps for the Hamiltonian with
 * eps V added to its Fock matrix (orbitals unrelaxed, as the response functions), at the
 * operators and frequencies of the last cc_lr_solve; d alpha / d eps = -out.  V: an n x n matrix,
 * row-major, host or device memory.  The derivative follows from the chain rule through the
 * ground amplitudes (t^V = -A^-1 xi^V), the multipliers (lam^V A = -(eta^V + F t^V)) and the
 * response amplitudes, whose derivatives are eliminated with the first-order multipliers
 * tbar^k(w) (A + w) = -(eta^k + F t^k(w)); the amplitude derivatives of sigma, xi, eta and F are
 * taken from the library's products at shifted amplitudes by stencils that are exact for their
 * polynomial degree.  Costs one right and one left static solve, 4 n_ops left solves per
 * frequency (solved together, each system holding 2 max_subspace vectors of N complex values),
 * and per frequency four Hbar builds with batched sigma and Hessian products.
 * Requires cc_lr_solve; CCLR_E_ARG on non-finite V; CCLR_E_NOCONV if a solve does not converge
 * (the context's amplitudes and multipliers are restored in every case). */
cclr_status cclr_field_derivative(cclr_ctx *ctx, const cclr_c128 *V, cclr_c128 *out);

/* EOM-CCSD excitation energies (SI "EOM-EE sigma-vectors and intermediates"; the Davidson scheme
 * applied to the eigenproblem): the n_roots (1..16) eigenvalues of the CC Jacobian A with the
 * smallest real part, from a non-Hermitian Davidson iteration on right sigma products with the
 * orbital-energy-denominator preconditioner.  energies_out receives n_roots complex values (the
 * real part is the excitation energy in Hartree), ordered by real part; iters_out (may be NULL)
 * the iteration count.  Options: tol (absolute residual norm of the unit right vector),
 * max_subspace, maxit, batch, precision (tensor-core modes stop at 1e-5 |w|).  Requires
 * cc_ground (CCLR_E_STATE); CCLR_E_NOCONV if maxit is reached. */
cclr_status cc_eom_ee(cclr_ctx *ctx, int n_roots, cclr_c128 *energies_out, int *iters_out);

/* Right eigenvector of root `root` of the last cc_eom_ee in the amplitude layout (n = o*v + Po*Pv
 * values, host buffer, norm 1 over the unique excitations to the solver's precision). */
cclr_status cclr_get_eom_vector(cclr_ctx *ctx, int root, cclr_c128 *dst, size_t n);

/* ---------------- component entry points (parity tests, the autograd shim) ------------------ */

/* Which amplitude set: ground T, Lambda, or a response solution. */
enum { CCLR_AMP_T = 0, CCLR_AMP_LAMBDA = 1 };

/* Caller arrays of amplitudes, operators, right-hand sides and gradients (cclr_get/set_amplitudes,
 * cclr_get_response_vector, cclr_residual, cclr_xi, cclr_eta, cclr_eta_ground, cc_lr_solve's ops,
 * cclr_left_solve, cclr_response_gradient, cclr_get_eom_vector) may be host memory or device
 * memory: with unified addressing the copy direction follows from the pointer.  The calls return
 * after their copies complete; the caller orders device inputs before the call (e.g. by
 * synchronizing the stream that wrote them). */

/* Copy amplitudes out in the amplitude layout (n must be o*v + Po*Pv). */
cclr_status cclr_get_amplitudes(cclr_ctx *ctx, int which, cclr_c128 *dst, size_t n);

/* Set T (and rebuild the Hbar intermediates) or Lambda from host data in the amplitude layout,
 * bypassing cc_ground / cc_lambda (used to test contractions at arbitrary amplitudes). */
cclr_status cclr_set_amplitudes(cclr_ctx *ctx, int which, const cclr_c128 *src, size_t n);

/* Response solution t^X(z) for operator k, frequency f and shift s (0: w+ig, 1: -w+ig,
 * 2: w-ig, 3: -w-ig) after cc_lr_solve, in the amplitude layout. */
cclr_status cclr_get_response_vector(cclr_ctx *ctx, int k, int f, int s, cclr_c128 *dst, size_t n);

/* One export call for every amplitude set: which = 0 the ground amplitudes T, 1 the multipliers
 * Lambda (idx ignored; as cclr_get_amplitudes), 2 a response solution t^X(z) with
 * idx = (k * n_freq + f) * 4 + s (as cclr_get_response_vector).  n must be o*v + Po*Pv. */
cclr_status cclr_export_amplitudes(cclr_ctx *ctx, int which, int idx, cclr_c128 *dst, size_t n);

/* Sigma vectors for nvec vectors in the amplitude layout (side 0: right, A r, SI Eqs.
 * sigma_sin-ee / sigma_double-ee; side 1: left, l A, SI Eqs. sigma_sin-ee-left /
 * sigma_double-ee-left).  on_device != 0 means `in` and `out` are device pointers on the
 * context's device (e.g. from torch tensors); otherwise host pointers.  Uses the current T
 * (and its Hbar).  precision selects the contraction arithmetic (cclr_precision). */
cclr_status cclr_sigma(cclr_ctx *ctx, int side, int nvec, const cclr_c128 *in, cclr_c128 *out,
                       int on_device, int precision);

/* CCSD residual Omega(T) at the current T (amplitude layout, host). */
cclr_status cclr_residual(cclr_ctx *ctx, cclr_c128 *out, cclr_c128 *e_corr_out);

/* xi^X (SI Eq. xi-equation), eta^X (SI Eq. eta-equation) and, with eom != 0, the EOM eta^X of
 * the SI, for one Hermitian operator X (host (o+v)^2).  eta needs Lambda.  These and
 * cclr_hessian compute in the precision of the response results: FP64-class tensor cores
 * (CCLR_TC_F64) on a split-BF16 context that refines, the context's precision otherwise. */
cclr_status cclr_xi(cclr_ctx *ctx, const cclr_c128 *op, cclr_c128 *out);
cclr_status cclr_eta(cclr_ctx *ctx, const cclr_c128 *op, int eom, cclr_c128 *out);

/* CC Hessian products (u F) (SI, "(t^X F)" working equations) for nvec vectors; needs Lambda. */
cclr_status cclr_hessian(cclr_ctx *ctx, int nvec, const cclr_c128 *u, cclr_c128 *out, int on_device);

/* The contraction engine's GEMM on its own (used to test the tensor-core kernels):
 *   C[m][n] = sum_k A[m][k] B[n][k]  (complex, row-major, both operands K-major, host pointers,
 *   A: M x K, B: N x K, C: M x N), in the given precision.  Needs a Hamiltonian (for the
 *   context's device workspace). */
cclr_status cclr_zgemm_nt(cclr_ctx *ctx, int precision, int M, int N, int K, const cclr_c128 *A,
                          const cclr_c128 *B, cclr_c128 *C);

/* The Davidson solver's Gram block on its own (parity tests): out[i*ny + j] = sum_k conj(X_i[k]) Y_j[k]
 * for host row-major X (nx x n) and Y (ny x n), computed by the FP32-arithmetic kernel the
 * tensor-core modes use, from FP64 rows (mirror = 0) or from FP32 copies with even row strides
 * (mirror = 1, the solver's trial-vector mirrors).  Needs a Hamiltonian (device workspace). */
cclr_status cclr_gram(cclr_ctx *ctx, int mirror, int64_t n, int nx, int ny, const cclr_c128 *X, const cclr_c128 *Y,
                      cclr_c128 *out);

/* The Davidson solver's multi-vector kernels on their own (measurement; the paper's Davidson
 * scheme, SI "Davidson scheme", does these passes over the trial vectors every iteration).
 * On nx + max(ny, m) synthetic device vectors of length n (deterministic values, allocated and
 * freed here), after one warm-up call each, times `reps` calls of
 *   ms3[0]  the Gram block X^H Y (nx x ny),
 *   ms3[1]  Y_q = sum_j X_j C_jq for m outputs, squared norms only (the residual-norm pass),
 *   ms3[2]  the same with the m outputs stored (the correction pass),
 * and returns milliseconds per call (CUDA events on the context's stream).  The arithmetic is
 * the solver's for that precision: FP32 pairs in the mixed modes (CCLR_TC_BF16X3, BF16X6),
 * float-float in CCLR_FP64 and CCLR_TC_F64 (the refinement's passes).  1 <= m <= 16, nx <= 512.
 * Needs a Hamiltonian (for the context's workspace). */
cclr_status cclr_bench_vector_kernels(cclr_ctx *ctx, int precision, int64_t n, int nx, int ny, int m, int reps,
                                      double *ms3);

/* Allocation-free tensor-core GEMM (the paper has no counterpart; it serves callers that cannot
 * allocate device memory: a framework that owns all device memory through its own pool, a
 * server that fixes its footprint after start-up, or code running where an allocation may block).
 *   C[m][n] = sum_k A[m][k] B[n][k]   complex, row-major, DEVICE pointers on the current device,
 *   A: M x K, B: N x K, C: M x N (written, not accumulated); precision CCLR_TC_BF16X3 or
 *   CCLR_TC_BF16X6 (same slicing and kernel as the context's tensor-core contractions).
 * No context, and no cudaMalloc / cudaFree or allocating library call: every temporary (BF16
 * operand slices, split-K partial tiles, the kernel's status word) lives in one fixed 64 MiB
 * file-scope device array that each device holds from library load until process exit.
 * Sizes whose temporaries exceed it return CCLR_E_ARG with no GPU work (a square problem fits up
 * to M = N = K of about 1000 with three products).  stream may be NULL (legacy default stream); the call
 * is synchronous: it reads the status word back and synchronizes the stream before it returns.
 * The first call on a device resolves the array's device address with that device current; make
 * that first call before any stream capture.  Every
 * call shares the array and each call clears the status word it uses, so calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialized by the caller.
 * Returns CCLR_E_TIMEOUT if a bounded device wait expired, CCLR_E_CUDA on a runtime error. */
cclr_status cclr_zgemm_nt_noalloc(int precision, int M, int N, int K, const cclr_c128 *A, const cclr_c128 *B,
                                  cclr_c128 *C, void *stream);

/* Timing of the tensor-core GEMM kernels with CUDA events recorded on the context's stream around
 * every launch.  enable != 0 switches recording on.  out8 (may be NULL) receives, accumulated
 * since the previous call, for the split-BF16 kernel (out8[0..3]) and the FP64-class kernel
 * (out8[4..7]): {launches, milliseconds, executed BF16 flops (8 M N K per slice or digit
 * product), useful complex flops (8 M N K)}; the counters are then reset. */
cclr_status cclr_kernel_profile(cclr_ctx *ctx, int enable, double *out8);

/* Per-kernel timing switched on by cclr_kernel_profile: a pair of CUDA events on the context's
 * stream around every launch of the library, summed per kernel name.  Writes one text line per
 * kernel, "name launches milliseconds\n", most expensive first, into buf (cap bytes including
 * the terminating NUL; longer text is truncated) and resets the totals.  The library's own
 * measurement aid, not an operation of the paper.  CCLR_E_ARG if buf is NULL or cap < 1. */
cclr_status cclr_kernel_breakdown(cclr_ctx *ctx, char *buf, int cap);

/* Test of the failure path of the tensor-core GEMM's bounded waits (not an operation of the
 * paper): the next launch of the split-BF16 GEMM kernel on this context waits first for a
 * barrier phase that nothing completes, with a limit of `polls` polls (about 256 ns each) on
 * every wait, so the wait runs out before any copy or MMA is issued; the kernel records the
 * expiry, every role exits, TMEM is freed, and the call that launched it returns CCLR_E_TIMEOUT.
 * The context stays usable.  CCLR_E_ARG for polls = 0. */
cclr_status cclr_debug_expire_next_wait(cclr_ctx *ctx, unsigned polls);

/* Several systems of uneven size solved as one batch: for every k < n, context ctxs[k] (its own
 * Hamiltonian, set by cclr_set_hamiltonian, and its own stream) runs cc_ground, cc_lambda,
 * cc_lr_solve(n_ops operators ops[k], the n_freq frequencies omegas, gamma) and
 * cc_response_function into out[k] (n_freq*n_ops*n_ops values), each system on its own host
 * thread, so that the kernels of the systems overlap on the GPU (the GEMMs of a small system
 * occupy few SMs).  The contexts must be distinct; each call is as documented for one context.
 * status (may be NULL) receives each system's status; the return value is the first non-OK
 * status in system order, CCLR_OK if all succeeded, CCLR_E_ARG for bad arguments. */
cclr_status cclr_response_batch(cclr_ctx *const *ctxs, int n, int n_ops, const cclr_c128 *const *ops, int n_freq,
                                const double *omegas, double gamma, cclr_c128 *const *out, cclr_status *status);

/* The tile autotuner's decisions so far, one text line per GEMM shape: "MxNxK/slices/c|s/SMs rows
 * stages ms_128 ms_64" (the shape key, the chosen tile rows and pipeline stages, and the timed
 * milliseconds of the two candidates), into buf (cap bytes including the terminating NUL; longer
 * text is truncated).  CCLR_E_ARG if buf is NULL or cap < 1. */
cclr_status cclr_autotune_report(cclr_ctx *ctx, char *buf, int cap);

/* Per-call statistics of the last cc_* call: sigma launches and vectors, seconds spent;
 * refine_vectors / refine_seconds: the FP64-class sigma products (CCSD residuals) and the
 * seconds of the refinement phase; max_residual: the largest final residual norm. */
typedef struct {
  long sigma_calls, sigma_vectors;
  double sigma_seconds, total_seconds;
  long kernel_launches;
  double max_residual;
  long refine_vectors;
  double refine_seconds;
} cclr_stats;
cclr_status cclr_get_stats(cclr_ctx *ctx, cclr_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* CCLR_H */
