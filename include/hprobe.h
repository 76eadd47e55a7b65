/*
 * hprobe.h - C ABI of the GB300 hierarchical-probing library.
 *
 * Estimates Tr(A^-1) for lattice operators A on 4-D tori with the nested
 * Hadamard/Fourier probing vectors of Stathopoulos, Laeuchli and Orginos,
 * "Hierarchical probing for estimating the trace of the matrix inverse on
 * toroidal lattices" (arXiv:1302.4018).  Every step runs in CUDA kernels
 * compiled for sm_103a; the host code only validates, schedules and copies.
 *
 * Conventions shared by every call
 *   - Sites are numbered lexicographically, x_1 fastest:
 *       site = x_1 + L_1 (x_2 + L_2 (x_3 + L_3 x_4)).
 *   - Unknown (spin s, colour c) of a Wilson site is 12 * site + 3 s + c.
 *   - Buffers marked "host or device" may be either: the library asks the
 *     CUDA driver which one it is and copies host data itself.  Buffers
 *     marked "device" must be device memory of the context's GPU.
 *   - The caller owns and allocates every input and output; the library
 *     never frees caller memory.  Workspace belongs to the context.
 *   - Work is ordered on the context's stream.  Calls that return host
 *     results synchronise that stream before returning.
 *   - No call aborts, throws or exits: each returns an hp_status and, on
 *     failure, hp_last_error() describes the cause (per calling thread).
 */
#ifndef HPROBE_H
#define HPROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HP_OK = 0,
    HP_EINVAL = 1,        /* an argument is out of range or inconsistent          */
    HP_EUNSUPPORTED = 2,  /* valid request the method cannot serve (see below)   */
    HP_ENOMEM = 3,        /* device or pinned-host allocation failed             */
    HP_ECUDA = 4,         /* a CUDA runtime call failed                          */
    HP_ENOCONV = 5,       /* some right-hand side missed tol within maxiter      */
    HP_ETIMEOUT = 6       /* a bounded device wait gave up                       */
} hp_status;

typedef struct hp_ctx hp_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on (NULL: the context creates its own blocking stream, which is
 * ordered with the legacy default stream).  Device inputs must be ready in
 * that stream order, and device outputs are ready in that order.
 * On success *out owns device workspace until hp_ctx_destroy. */
hp_status hp_ctx_create(int device, void* cuda_stream, hp_ctx** out);
void hp_ctx_destroy(hp_ctx* ctx);
/* Message of the last failed call on this thread (never NULL). */
const char* hp_last_error(void);
/* Wait for all work queued on the context's stream. */
hp_status hp_ctx_synchronize(hp_ctx* ctx);

/* A lattice: ndim in [1, 8] sizes; operators need ndim <= 4 (missing
 * dimensions are size 1).  The volume must be at most 2^31. */
typedef struct {
    int32_t ndim;
    int64_t dims[8];
} hp_lattice;

/* Facts about the probing basis of a lattice (Sections 2.2, 3.3, 3.4).
 * L_j = 2^{k_j} p_j with p_j odd; K = sum k_j binary levels; Q = prod p_j.
 * When Q > 1 the three-colour level (theorem of Section 3.4) follows the
 * binary levels; if its three classes are equal (R = Q / 3 each) a final
 * dense Fourier level of size R completes the basis, otherwise only the
 * first 2^K vectors exist (Section 2.2: no nested basis for unequal colour
 * counts).  Entries of every vector are exp(2 pi i phase / period). */
typedef struct {
    int64_t volume;
    int64_t n_vectors;       /* vectors of the nested sequence available        */
    int32_t K, Q, R;         /* R = 0 when the odd classes are unequal          */
    int32_t period;          /* P: common period of all phases (even)           */
    int32_t kmax;
    int32_t ks[8], ps[8];
} hp_basis;

hp_status hp_basis_info(const hp_lattice* lat, hp_basis* out);

/* The value table of the phases: out[2k], out[2k+1] = cos, sin of 2 pi k / P
 * for k = 0 .. P-1 (host array of 2P doubles), each rounded once to binary64
 * from a double-double evaluation after an exact octant reduction.  These
 * are the entries exp(2 pi i k / P) of the Fourier matrices of Eq.
 * (FourierElements) used by the device.  Host-only; needs no GPU.
 * Errors: HP_EINVAL for P < 1 or P > 65535 or out == NULL. */
hp_status hp_phase_values(int32_t period, double* out);

/* Hierarchical permutation (Section 3, Algorithm 5 with the closed form of
 * the red-black table from the third lemma of Section 3.3, then the
 * three-colour level of Section 3.4 for odd factors).
 * loc_dev[site] (device, uint32[V]) receives the 0-based position of the
 * site in the hierarchical order, i.e. the inverse permutation "iperm" of
 * Section 2.1.  The binary levels give the most significant digits; inside
 * a level dimension 1 gives the most significant bit.
 * Errors: HP_EINVAL for ndim outside [1,8], a size < 1 or V > 2^31. */
hp_status hp_permutation(hp_ctx* ctx, const hp_lattice* lat, uint32_t* loc_dev);

/* Probing vectors v_m = z_0 (.) z_m for m = first .. first+count-1 (Section 2.2,
 * Eq. row-col-permutation generalised to Eq. Hperm-general-recursive, and
 * Section 4, Eq. removebias).  phase_dev (device, uint16[count][V]) receives
 * phase[j * V + site] with v_{first+j}(site) = exp(2 pi i phase / P);
 * *period_out (host) receives P.  z0_seed == 0 means z_0 = 1; otherwise
 * z_0(site) = -1 iff the top bit of output number `site` (0-based) of
 * Vigna's SplitMix64 generator seeded with z0_seed is set.
 * Errors: HP_EINVAL for first < 0, count < 0 or first+count > V;
 * HP_EUNSUPPORTED when first+count exceeds n_vectors (unequal odd classes). */
hp_status hp_probe_vectors(hp_ctx* ctx, const hp_lattice* lat, int64_t first, int64_t count,
                           uint64_t z0_seed, uint16_t* phase_dev, int32_t* period_out);

typedef enum { HP_OP_LAPLACIAN = 0, HP_OP_WILSON = 1 } hp_op_kind;

/* The operator A (Section 5: shifted periodic Laplacian; Section 1.1.1 and
 * 5.3: Wilson-Dirac matrix, with the clover term of the Clover-Wilson
 * discretisation Section 5.3 uses when csw != 0).
 *   Laplacian:  (A x)(s) = (8 + mass + mu(s)) x(s) - sum_mu [x(s+mu) + x(s-mu)]
 *   Wilson:     (D psi)(s) = (1 + mass + mu(s)) psi(s) + C(s) psi(s)
 *                 - kappa sum_mu [(1 - g_mu) U_mu(s) psi(s+mu) + (1 + g_mu) U_mu(s-mu)^H psi(s-mu)]
 *     chiral gamma basis: g_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1..3),
 *     g_4 = [[0, 1], [1, 0]], g_5 = diag(1, 1, -1, -1); direction mu = k runs along x_k.
 *     Clover (Sheikholeslami-Wohlert) term:
 *       C(s) = -csw kappa sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(s),  sigma_{mu nu} = (i/2)[g_mu, g_nu],
 *       F_{mu nu} = traceless part of (Q_{mu nu} - Q_{mu nu}^H) / (8i), Q_{mu nu}(s) the four
 *       plaquettes of the mu-nu plane that start and end at s, each run mu-then-nu.
 * links: Wilson only, complex128 [V][4][3][3] (row-major 3x3 per site and
 *        direction, real/imaginary interleaved), host or device, special unitary.
 * mass_field: optional mu(s), double[V], host or device; NULL means 0.
 * csw: clover coefficient, Wilson only (0: plain Wilson; the Laplacian requires 0);
 *      the 12x12 diagonal blocks 1 + mass + mu(s) + C(s) must be invertible. */
typedef struct {
    int32_t kind;
    double mass;
    double kappa;
    const double* links;
    const double* mass_field;
    double csw;
} hp_operator;

typedef enum {
    HP_PREC_FP64 = 0,        /* everything in FP64                                       */
    HP_PREC_MIXED_FP32 = 1,  /* FP32 iteration, FP64 reliable updates / true residual   */
    HP_PREC_MIXED_FP16 = 2,  /* FP16 storage (per-site norm) with FP32 arithmetic inside */
    HP_PREC_MIXED_BF16 = 3   /* BF16 storage (per-site norm) with FP32 arithmetic inside */
} hp_precision;

/* The probing sequence: hierarchical probing (Sections 2-4, the default) or one of the two
 * sequences Section 5.2 compares it with: Hadamard vectors in natural order, z_m(s) = H_V(s, m)
 * (Sylvester matrix, lexicographic sites, V a power of two, bias removed with z_0 as for
 * hierarchical probing), and independent Z_2 noise vectors, z_m(s) = -1 iff the top bit of
 * output number m V + s of SplitMix64 seeded with z0_seed is set (the standard Monte Carlo
 * estimator of Section 1.1.2).  Errors: HP_EUNSUPPORTED for natural order on a V that is not a
 * power of two; HP_EINVAL for an unknown kind. */
typedef enum { HP_PROBE_HIERARCHICAL = 0, HP_PROBE_NATURAL = 1, HP_PROBE_Z2 = 2 } hp_probe_kind;

/* hp_probe_vectors for any hp_probe_kind (kind 0 is hp_probe_vectors itself): the phases of
 * v_m, m = first .. first+count-1, as uint16[count][V] on the device with P = *period_out (the
 * lattice's period; the natural and Z_2 sequences use the phases 0 and P/2 only).
 * Errors as hp_probe_vectors, plus HP_EINVAL for an unknown kind and HP_EUNSUPPORTED for
 * natural order on a V that is not a power of two. */
hp_status hp_probe_sequence(hp_ctx* ctx, const hp_lattice* lat, int32_t kind, int64_t first, int64_t count,
                            uint64_t z0_seed, uint16_t* phase_dev, int32_t* period_out);

typedef struct {
    int32_t precision;      /* hp_precision                                              */
    int32_t rhs_block;      /* right-hand sides solved concurrently (0: automatic)       */
    int32_t maxiter;        /* iterations per right-hand side (0: 10000)                 */
    int32_t dilution;       /* 12 for Wilson (full spin-colour dilution), 1 for Laplacian; 0: default */
    uint64_t z0_seed;       /* bias-removal vector, 0 = none (Section 4)                 */
    int64_t first;          /* first probe to solve; q of probes < first come from q_inout */
    double delta;           /* group-update threshold on ||r||/max||r|| (0: per precision:
                               0.001 FP32, 0.03 FP16/BF16, measured on the 32^3x64 workload) */
    int32_t check_every;    /* iterations between host scheduling steps (0: automatic)   */
    int32_t use_graph;      /* 1: replay the iteration chunk from a captured CUDA graph  */
    int32_t block_threads;  /* reserved for the stencil block size (0)                    */
    int32_t rhs_per_thread; /* stencil variant: 1, 2, 4 right-hand sides per thread with 12-real
                               links, + 100 for 18-real links, + 1000 G to sweep the lattice
                               in groups of G slots (0: autotune)                           */
    int32_t even_odd;       /* Wilson: 1 = iterate on the odd-site Schur complement
                               d_o - kappa^2 H_oe d_e^-1 H_eo (needs every extent even, the
                               lattice padded to four dimensions included, else the full
                               lattice is iterated; the certified
                               residual is still that of the full system)                   */
    int32_t probe_kind;     /* hp_probe_kind: the probing sequence (0: hierarchical probing) */
    int32_t eo_kernel;      /* even-odd iteration in FP32 / FP16 / BF16: the V and T step kernels --
                               1 one right-hand side per thread; 3, 4 two right-hand sides per
                               thread (packed FP32x2 arithmetic) with 3 or 4 resident blocks of 128
                               threads per SM; 13, 14 the same with FP32 links; 5 the two-sided
                               even-site kernel with the one-sided odd-site kernel; 6 the even-site
                               hop on the tensor cores (mma.sync, FP16 x FP16 -> FP32; FP16
                               iterations of one lattice without the clover term, up to 32 slots,
                               else 0) with the two-sided odd-site kernel -- slower than 4 on GB300
                               and never the autotuner's choice; 0: the fastest of 1, 3, 4, 5, 13,
                               14, timed on the problem's largest lattice and cached in the context */
    int32_t reserved[1];
} hp_solver_opts;

typedef struct {
    int64_t rhs_solved;
    int64_t iterations_total;     /* sum over right-hand sides                         */
    int32_t iterations_max;
    int32_t iterations_min;
    int64_t reliable_updates;     /* FP64 true-residual recomputations                 */
    int64_t sloppy_matvecs;       /* per right-hand side, iteration precision          */
    int64_t fp64_matvecs;         /* per right-hand side, FP64                         */
    double max_true_residual;     /* max ||b - A x|| / ||b|| in FP64 at convergence    */
    double seconds;               /* wall time of the call                             */
    int32_t n_unconverged;
    int32_t group_updates;        /* FP32 group updates of x and r between FP64 ones   */
} hp_solve_stats;

/* The incremental trace estimate (Section 1: (1/s) sum_k z_k^H A^-1 z_k;
 * Section 1.1.2: each quadrature by a linear solve; Section 2.2: nested
 * prefixes; Section 5.3: full spin-colour dilution for Wilson).
 * For probe m and dilution index a the source is v_{m,a} = (z_0 (.) z_m) (x) e_a
 * (Wilson; the Laplacian has one source per probe, split into real and
 * imaginary parts when the probe is complex), solved to a TRUE relative
 * residual ||b - A x||_2 / ||b||_2 <= tol computed in FP64.
 *   q_m = sum_a v_{m,a}^H x_{m,a},   T_s = (1/s) sum_{m<s} q_m.
 * q_inout (host, nullable): complex q[m] as (re, im) pairs for m < s_max;
 *   entries m < opts->first are inputs (an earlier run), the others outputs.
 * trace_prefix (host): (re, im) of T_s at [2 (s-1)], s = 1 .. s_max.
 * stats (host, nullable).
 * Errors: HP_EINVAL (s_max < 1, first outside [0, s_max), tol <= 0, bad
 * operator fields, ndim > 4 for operators); HP_EUNSUPPORTED (s_max above
 * n_vectors); HP_ENOCONV when a right-hand side misses tol in maxiter
 * (outputs still filled from the last iterate). */
hp_status hp_trace_inv(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                       double tol, const hp_solver_opts* opts, double* q_inout, double* trace_prefix,
                       hp_solve_stats* stats);

/* hp_trace_inv that also returns the solutions x_{m,a} of the first n_keep
 * right-hand sides it solves (Wilson only): right-hand side j = 12 (m - first) + a
 * of x_out (device, complex128 [n_keep][V][4][3] in the canonical layout of
 * hp_operator_apply) receives the converged A^-1 v_{m,a} as the solver holds it
 * (FP64, or the float-float solution of the mixed modes rounded to FP64).
 * With them a caller checks ||v_{m,a} - A x_{m,a}|| / ||v_{m,a}|| and
 * q_m = sum_a v_{m,a}^H x_{m,a} independently of the library (Section 1.1.2:
 * each quadrature is a linear solve).  n_keep = 0 is hp_trace_inv.
 * Errors: as hp_trace_inv, plus HP_EINVAL for a Laplacian, n_keep outside
 * [0, 12 (s_max - first)] or x_out not device memory. */
hp_status hp_trace_inv_solutions(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                                 double tol, const hp_solver_opts* opts, int64_t n_keep, double* x_out,
                                 double* q_inout, double* trace_prefix, hp_solve_stats* stats);

/* The prefix estimates of a quadrature sequence computed elsewhere (Section 1:
 * T_s = (1/s) sum_{m<s} q_m; Section 2.2: nested prefixes): q (host or device,
 * complex (re, im) pairs [s_max]) -> trace_prefix (host or device, the same
 * layout), summed in the order and FP64 arithmetic hp_trace_inv uses.  Ranks
 * that solved disjoint probe blocks gather their q into one sequence and call
 * this, so that their T_s equals a one-rank run's bit for bit.
 * Errors: HP_EINVAL for s_max outside [1, 2^31) or a NULL array. */
hp_status hp_trace_prefix(hp_ctx* ctx, int64_t s_max, const double* q, double* trace_prefix);

/* hp_trace_inv for the Hermitian positive definite Laplacian with guaranteed
 * bounds on every quadrature (Section 1.1.2: the Gauss quadrature of
 * z^H A^-1 z computed by Lanczos comes with lower and upper bounds): with
 * x_0 = 0, CG's step lengths gamma_k and residual ratios delta_{k+1} give the
 * Gauss rule G_k = sum_{j<k} gamma_j ||r_j||^2 <= z^H A^-1 z and, for a node
 * 0 < mu <= lambda_min(A), the Gauss-Radau rule G_k + gt_k ||r_k||^2 >= z^H A^-1 z,
 * gt_0 = 1/mu, gt_{k+1} = (gt_k - gamma_k) / (mu (gt_k - gamma_k) + delta_{k+1}).
 * Each solve stops when its bracket is at most quad_tol times G_k (no residual
 * test: the bracket certifies the quadrature, whose error falls as the square
 * of the residual).  lambda_min: the node mu; <= 0 selects mass + min mu(s)
 * (the hopping part of A is positive semidefinite).
 * trace_prefix (host): T_s from z^H x as in hp_trace_inv; T_lower, T_upper
 * (host, double[s_max]): bounds on Re T_s, s = 1 .. s_max.  opts->first must be 0.
 * Errors: HP_EINVAL for a Wilson operator, quad_tol <= 0, a node <= 0; as
 * hp_trace_inv otherwise (HP_ENOCONV if a bracket does not close in maxiter). */
hp_status hp_trace_inv_bounds(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                              double quad_tol, double lambda_min, const hp_solver_opts* opts,
                              double* trace_prefix, double* T_lower, double* T_upper, hp_solve_stats* stats);

/* Deflated hierarchical probing: the variance reduction that the paper's
 * conclusions name as the next step after probing.
 *
 * Laplacian (real symmetric positive definite).  With k orthonormal real eigenvectors V of A
 * (evecs: double[k][V] in the canonical site order, host or device) and their
 * eigenvalues (evals: host double[k], all > 0), P = I - V V^T and
 *   Tr A^-1 = sum_j 1/lambda_j + Tr(A^-1 P),
 * the second term is estimated by probing with the projected vectors
 * P v_m (v_m as in hp_trace_inv):
 *   q_m = (P v_m)^H A^-1 (P v_m),  T_s = sum_j 1/lambda_j + (1/s) sum_{m<s} q_m.
 * The identity needs V to span an invariant subspace (eigenvectors): other
 * vectors give a biased estimate.  Removing the lowest modes removes the long-
 * range part of A^-1 that the colouring cannot, so T_s converges faster.
 *
 * Wilson.  With k orthonormal eigenvectors w_j of the Hermitian Q = gamma_5 D
 * (gamma_5-hermiticity; evecs: complex double[k][V][4][3], host or device) and
 * their real eigenvalues lambda_j (host double[k], non-zero; hp_wilson_eigs
 * computes them), the left vectors u_j = gamma_5 w_j are orthonormal and
 * D^-1 u_j = w_j / lambda_j, so
 *   Tr D^-1 = sum_j (w_j^H gamma_5 w_j) / lambda_j + Tr(D^-1 (I - U U^H)),
 * and the second term is probed: q_m = sum_a v_{m,a}^H D^-1 (I - U U^H) v_{m,a}.
 * The solves are the plain ones of hp_trace_inv (any precision and options);
 * each quadrature is then corrected on the device by
 *   - sum_a gamma_5(a) sum_j |v_{m,a}^H w_j|^2 / lambda_j,
 * whose projections of the first s_max vectors onto the w_j follow from sums
 * of the w_j over the blocks of hierarchical positions the vectors are
 * constant on (Walsh-Hadamard sums; every position its own block past the
 * binary levels).  Hierarchical vectors only (probe_kind 0).
 *
 * q_inout (the deflated quadratures), trace_prefix, stats as hp_trace_inv;
 * opts->first must be 0.  Errors: HP_EINVAL for k outside [1, V] (Laplacian)
 * or [1, min(12 V, 65535)] (Wilson), NULL arrays, a Laplacian eigenvalue <= 0 or a Wilson
 * eigenvalue 0; HP_EUNSUPPORTED for another probe kind (Wilson); as
 * hp_trace_inv otherwise. */
hp_status hp_trace_inv_deflated(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k,
                                const double* evecs, const double* evals, int64_t s_max, double tol,
                                const hp_solver_opts* opts, double* q_inout, double* trace_prefix,
                                hp_solve_stats* stats);

/* Deflated probing of the Wilson matrix with singular triplets D v_j = sigma_j
 * u_j (right vectors v_j and left vectors u_j, each set orthonormal, complex
 * double[k][V][4][3], host or device; sigma host double[k], all > 0;
 * hp_wilson_svd computes them): D^-1 u_j = v_j / sigma_j, so
 *   Tr D^-1 = sum_j (u_j^H v_j) / sigma_j + Tr(D^-1 (I - U U^H)),
 * the second term probed with the plain solves and the correction
 *   - sum_a sum_j (v_{m,a}^H v_j) (u_j^H v_{m,a}) / sigma_j
 * of each quadrature, as in hp_trace_inv_deflated (whose gamma_5 eigenpairs are
 * the triplets v = w, u = sign(lambda) gamma_5 w, sigma = |lambda|).  The
 * identity holds for any singular triplets, so the k smallest need not sit at a
 * gap of the spectrum; it needs only D^-1 u_j = v_j / sigma_j, so it also holds
 * for the Rayleigh-Ritz triplets hp_wilson_svd returns before it converges.
 * Arguments and errors as hp_trace_inv_deflated for the Wilson operator
 * (HP_EINVAL also for a Laplacian, NULL left vectors or a sigma <= 0). */
hp_status hp_trace_inv_deflated_svd(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k,
                                    const double* right, const double* left, const double* sigma, int64_t s_max,
                                    double tol, const hp_solver_opts* opts, double* q_inout, double* trace_prefix,
                                    hp_solve_stats* stats);

/* The k eigenpairs of Q = gamma_5 D (Wilson or Clover-Wilson; Hermitian by
 * gamma_5-hermiticity, real eigenvalues of either sign) with the smallest
 * |lambda| -- the smallest singular values of D, the modes hp_trace_inv_deflated
 * removes from the Wilson trace.  Chebyshev-filtered subspace iteration on
 * complex spinor blocks of b = 2k + 8 vectors: each sweep filters the
 * block with a degree-16 Chebyshev polynomial of Q^2 = D^H D (positive
 * semidefinite, the same eigenvectors) damping [largest Ritz value of Q^2 on
 * the block, top of the spectrum of Q^2: 24 Lanczos steps, the largest Ritz
 * value plus the last off-diagonal element, capped by ||D||^2 <= (|1 + m| +
 * max |mu| + 16 kappa + 12 csw kappa)^2], orthonormalises it (Cholesky QR), and takes the
 * Rayleigh-Ritz pairs of Q^2 on the block, then those of Q inside the span of
 * the k lowest (Q is indefinite: its Ritz values on a block that mixes both
 * ends of the spectrum can fall anywhere, near 0 included); k should sit at a
 * gap of |lambda| (a +-pair of nearly equal |lambda| split by k converges
 * slowly).  FP64 Rayleigh-Ritz steps and residuals (the FP64 Wilson stencil,
 * complex Gram matrices and block rotations on the device; b x b Hermitian
 * Cholesky and Jacobi on the host); the filter runs the FP32 stencil until the
 * largest residual falls to max(1e-5, 100 tol) or stops falling (less than 10%
 * per sweep once below 1e-2), the FP64 one after.  Sized for
 * small lattices: on 16^4 and larger the lowest modes are too dense for the
 * degree-16 filter to separate in a reasonable number of sweeps (HP_ENOCONV;
 * measured: 16^4, k = 24, residual 3.3e-3 after 200 sweeps); hp_wilson_svd
 * needs no +-pair of Q separated and converges there when k ends a cluster of
 * the spectrum.  Stops when ||Q w_j - lambda_j w_j|| <= tol |lambda_j|
 * for j < k, or after max_sweeps (0: 200; then HP_ENOCONV, outputs hold the
 * last iterate).  evecs: complex double[k][V][4][3] (host or device), w_j
 * orthonormal; evals (host double[k]): lambda_j ordered by |lambda_j|; resid
 * (host double[k], nullable): the relative residuals.  Errors: HP_EINVAL for a
 * Laplacian, k outside [1, min(6 V, 1024)] (the Rayleigh-Ritz steps diagonalise
 * (2k + 8)^2 matrices on the host), tol <= 0, NULL outputs. */
hp_status hp_wilson_eigs(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k, double tol,
                         int32_t max_sweeps, double* evecs, double* evals, double* resid);

/* The k smallest singular triplets D v_j = sigma_j u_j of the Wilson matrix
 * (Wilson or Clover-Wilson) from the same iteration as hp_wilson_eigs without
 * its second step: the Rayleigh-Ritz pairs of Q^2 = D^H D on the block are the
 * right vectors v_j and sigma_j^2, converged when ||Q^2 v_j - sigma_j^2 v_j|| <=
 * tol sigma_j^2 (about ||D|| / sigma_j times the relative residual of a pair of
 * Q, so a tol near 1e-9 is the counterpart of 1e-11 there and the FP64 floor is
 * reached sooner), and u_j = D v_j / sigma_j = gamma_5 (Q v_j) / sigma_j.  No +-pair
 * of gamma_5 D needs resolving, so this converges where the eigenpairs of Q do
 * not separate; the k-th value should still end a cluster of the spectrum
 * (the pairs near k converge at the rate set by the gap between sigma_k^2 and
 * the (2k + 9)-th value; measured on 16^4 at kappa 0.115, whose values come in
 * shells of 12 and 96: k = 12 in 3.6 s and k = 108 in 74 s to tol 1e-8, while
 * k = 24 stays near 1e-3).  right, left: complex double[k][V][4][3] (host or device);
 * sigma (host double[k]) ascending; resid (host double[k], nullable).  Errors as
 * hp_wilson_eigs (NULL left included).  On HP_ENOCONV the outputs hold the last
 * Rayleigh-Ritz triplets: v orthonormal, sigma_j^2 their Ritz values of Q^2,
 * u_j = D v_j / sigma_j (orthonormal as well, since V^H Q^2 V = diag(sigma^2));
 * only D^H u_j = sigma_j v_j is off by the residual.  hp_trace_inv_deflated_svd
 * needs no more than D v_j = sigma_j u_j, so deflation with an unconverged
 * result stays exact and unbiased; it removes less variance. */
hp_status hp_wilson_svd(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k, double tol,
                        int32_t max_sweeps, double* right, double* left, double* sigma, double* resid);

/* The k lowest eigenpairs of the shifted Laplacian (real symmetric positive
 * definite; mass field allowed): the eigenvectors hp_trace_inv_deflated removes
 * exactly (the paper's conclusions name deflation as the step after probing).
 * Chebyshev-filtered subspace iteration on a block of b = k + max(8, k/2)
 * vectors: each sweep applies the degree-12 Chebyshev polynomial in A that
 * damps [theta_b, lambda_max] (theta_b the block's largest Ritz value,
 * lambda_max = 16 + mass + max mu(s), Gershgorin), orthonormalises the block
 * (Cholesky QR, shifted once, then twice plain) and rotates it onto the Ritz
 * vectors (Rayleigh-Ritz); it stops when each of the k lowest pairs has
 * ||A v - lambda v|| <= tol lambda.  Everything is FP64; the start block is
 * seeded (the result is deterministic).  Vectors of an eigenvalue that repeats
 * across index k are one basis of a subspace the method does not fix.
 * evecs (host or device, double[k][V], lexicographic sites): orthonormal;
 * evals (host, double[k]): ascending; resid (host, nullable, double[k]): the
 * relative residuals reached.  max_sweeps <= 0: 200.
 * Errors: HP_EINVAL for a Wilson operator, k outside [1, min(V/2, 1024)] (the
 * Rayleigh-Ritz steps diagonalise b^2 matrices on the host), tol <= 0, NULL
 * outputs; HP_ENOCONV when max_sweeps pass first (outputs still written). */
hp_status hp_laplacian_eigs(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k, double tol,
                            int32_t max_sweeps, double* evecs, double* evals, double* resid);

/* hp_trace_inv plus the derivative of Re T_{s_max} with respect to the
 * per-site mass mu(s) (real):
 *   dT/dmu(s) = -(1/s_max) sum_{m,a} sum_c conj(y_{m,a}(s,c)) x_{m,a}(s,c),  y = A^-H v.
 * The adjoint solution comes from the forward one: the Laplacian is real
 * symmetric (y = x) and the Wilson matrix is gamma_5-hermitian,
 * D^-H = g_5 D^-1 g_5, so with full dilution y_{m,a} = g5_a g_5 x_{m,a}.
 * dT_dmu: double[V], host or device.  dT_dm (host): the uniform-mass
 * derivative sum_s dT/dmu(s).  opts->first must be 0. */
hp_status hp_trace_inv_grad(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                            double tol, const hp_solver_opts* opts, double* trace_prefix,
                            double* dT_dmu, double* dT_dm, hp_solve_stats* stats);

/* Many lattices (uneven sizes, masses, kappas) in one schedule: the
 * right-hand sides of every lattice share one set of solver slots, so each
 * kernel launch advances all lattices at once, and a slot that converges is
 * refilled with the next right-hand side of any lattice.
 * trace_prefix[i] (host) has 2 * s_max[i] doubles.  opts->first must be 0. */
hp_status hp_trace_inv_batch(hp_ctx* ctx, int32_t nlat, const hp_operator* ops, const hp_lattice* lats,
                             const int64_t* s_max, double tol, const hp_solver_opts* opts,
                             double* const* trace_prefix, hp_solve_stats* stats);

/* Hierarchical colouring of a general sparse matrix (Section 2.1, Algorithm 1).
 * Level 1 colours the graph of A greedily, rows in increasing index, each row
 * taking the smallest colour none of the already coloured rows of its CSR row
 * has (entries i -> i are ignored).  The rows of each colour form a block of the
 * next level, whose graph is the pattern of A_b(rows, :) A_b(:, rows) for the
 * block's graph A_b; a block recurses unless it got one colour or as many
 * colours as rows (a diagonal or dense block), and no level beyond max_levels
 * is coloured.  Within every block rows keep their index order, so the result
 * is the sequential algorithm's, bit for bit (computed as Jones-Plassmann
 * rounds with the row index as priority, all blocks of a level at once).
 * n: rows (>= 1); row_ptr int32[n+1] (row_ptr[0] = 0, non-decreasing),
 * col_idx int32[row_ptr[n]] in [0, n): the pattern of A, host or device, read only.
 * paths: int32[max_levels][n], host or device, written: paths[l][i] = colour of
 * row i at level l + 1, 0 at the levels below the one where its block stopped.
 * radices (host, int32[max_levels]): c(l + 1) = the largest colour count of a
 * block of level l + 1 (0 past *n_levels); *n_levels (host): levels coloured.
 * Working memory: the next level's graph, deduplicated through hash tables of
 * up to four times its two-hop candidate count (HP_ENOMEM if that fails).
 * Errors: HP_EINVAL for n < 1, max_levels outside [1, 32], NULL outputs, a
 * decreasing row_ptr or a column index outside [0, n). */
hp_status hp_sparse_coloring(hp_ctx* ctx, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                             int32_t max_levels, int32_t* paths, int32_t* radices, int32_t* n_levels);

/* Algorithm 1's own outputs from a colour hierarchy (Section 2.1): perm, the
 * order Colors2Perm leaves the rows in (the rows of one colour adjacent, level
 * after level inside every block, the original order inside a block that
 * stopped), and colorOffsets, the (start, end, level) record of every block
 * the recursion visits, in the order it visits them (0-based positions of
 * perm, end inclusive; the matrix itself is (0, n - 1, 1)).
 * paths / n_levels as hp_sparse_coloring returns them (int32[n_levels][n],
 * host or device; the colours of a block are 0 .. k - 1).  perm: int32[n],
 * host or device, perm[k] = the row at position k (NULL: not wanted).
 * offsets: int32[offsets_cap][3], host or device (NULL: count only);
 * *n_offsets (host) = the number of blocks, at most 2n - 1.  Under
 * hp_sparse_coloring's max_levels cap a block of the last coloured level
 * whose colouring splits it records its colour classes one level deeper,
 * where the recursion visits them and stops.  Computed on the GPU: the blocks
 * level by level from the paths, then stable radix sorts.  Errors: HP_EINVAL
 * for n < 1, n_levels outside [0, 32], no output, a colour outside [0, size of
 * its block), or more blocks than offsets_cap (*n_offsets then holds the
 * count). */
hp_status hp_sparse_ordering(hp_ctx* ctx, int32_t n, const int32_t* paths, int32_t n_levels, int32_t* perm,
                             int32_t* offsets, int64_t offsets_cap, int64_t* n_offsets);

/* The probing vectors of a colour hierarchy (Section 2.2, Eq. Hperm-general-
 * recursive, with the Fourier factor F_c(l) at every level): vector m has the
 * mixed-radix digits d_l(m) (radix c(l), level 1 least significant) and
 *   v_m(i) = z_0(i) prod_l exp(2 pi i d_l(m) paths[l][i] / c(l)),
 * z_0 as in hp_probe_vectors (none for z0_seed = 0).  Where blocks of one level
 * have different colour counts, c(l) is the largest (every row's colour is below
 * it), so the first c(1)...c(k) vectors are exactly orthogonal on each
 * colour class of level k.  The levels used are the smallest k with
 * c(1)...c(k) >= first + count; the phases (uint16[count][n], device) are
 * over the period P = lcm(2, c(1), ..., c(k)) returned in *period_out (host).
 * paths / radices / n_levels as hp_sparse_coloring returns them (paths host or
 * device; radices host).  Errors: HP_EINVAL for a range outside [0, n], a colour
 * outside [0, c(l)), a host phase_dev; HP_EUNSUPPORTED when the hierarchy
 * resolves fewer than first + count vectors or P exceeds 65535. */
hp_status hp_sparse_probe_vectors(hp_ctx* ctx, int32_t n, const int32_t* paths, const int32_t* radices,
                                  int32_t n_levels, int64_t first, int64_t count, uint64_t z0_seed,
                                  uint16_t* phase_dev, int32_t* period_out);

/* hp_trace_inv for a real symmetric positive definite sparse matrix A in CSR
 * (row_ptr, col_idx as hp_sparse_coloring; values double[row_ptr[n]]; host or
 * device): the probes are hp_sparse_probe_vectors' (opts->probe_kind 0) or the
 * natural-order Hadamard / Z_2 sequences (1, 2; paths unused), each solved by
 * CG to a true relative residual tol computed in FP64 (complex probes as two
 * real solves).  The right-hand sides run in blocks of B = 32, 64 or 128
 * (opts->rhs_block rounded up; 0: 64) with the vectors stored [row][B].
 * opts->precision: HP_PREC_FP64, or HP_PREC_MIXED_FP32 = FP32 iteration with
 * FP64 reliable updates (a true residual whenever ||r|| fell by opts->delta,
 * default 1e-5, since the last one).  q_inout, trace_prefix, stats as
 * hp_trace_inv.  Errors: as hp_trace_inv and hp_sparse_probe_vectors, plus
 * HP_EUNSUPPORTED for FP16 / BF16.  A matrix that is not symmetric positive
 * definite ends in HP_ENOCONV. */
hp_status hp_trace_inv_sparse(hp_ctx* ctx, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                              const double* values, const int32_t* paths, const int32_t* radices, int32_t n_levels,
                              int64_t s_max, double tol, const hp_solver_opts* opts, double* q_inout,
                              double* trace_prefix, hp_solve_stats* stats);

/* y = A x for nrhs fields in the canonical layout: Wilson complex128
 * [nrhs][V][4][3], Laplacian double [nrhs][V]; host or device.  precision
 * selects the stencil kernel used (the input is rounded to that storage,
 * the result returned in FP64). */
hp_status hp_operator_apply(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t nrhs,
                            int32_t precision, const double* in, double* out);

/* The operator the even-odd iteration solves (opts->even_odd = 1): with the
 * sites split by parity (x_1 + x_2 + x_3 + x_4 even / odd) the Wilson matrix is
 * [[A_e, -kappa H_eo], [-kappa H_oe, A_o]] (A = 1 + mass + mu(s) + C(s), the
 * site-diagonal part; H the hopping term of Section 1.1.1), and its odd-site
 * Schur complement is
 *     S = A_o - kappa^2 H_oe A_e^-1 H_eo.
 * out = S in on the odd sites (zero on the even sites) for nrhs fields in the
 * canonical layout of hp_operator_apply (host or device; the even sites of in
 * are ignored), computed by the kernels and the precision the iteration uses
 * (precision as hp_operator_apply: the input is rounded to that storage, the
 * result returned in FP64) and the kernel variant eo_kernel (as
 * hp_solver_opts.eo_kernel; 0 or an unknown value: the autotuner's choice;
 * FP64 has one variant).  Errors: HP_EINVAL for a Laplacian, an odd extent
 * or fewer than four dimensions (then some hop joins sites of one parity and
 * the split does not exist), kappa = 0, nrhs outside [1, 65532]. */
hp_status hp_schur_apply(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t nrhs,
                         int32_t precision, int32_t eo_kernel, const double* in, double* out);

/* y = D x for the Wilson operator in FP64, allocating nothing (the paper has
 * no counterpart: this serves callers that cannot let a library allocate GPU
 * memory, e.g. an application whose device memory is reserved up front by
 * another framework's allocator, or one that must keep synchronising
 * cudaMalloc / cudaFree calls off a latency-critical stream).
 * Same operator, layouts and FP64 arithmetic as hp_operator_apply with
 * HP_PREC_FP64; op->links, op->mass_field (nullable), in_dev and out_dev
 * must all be device memory of the current device, and out_dev must not
 * overlap in_dev, the links or the mass field (threads write a site's output
 * while others still read its neighbours' input, so an in-place call would
 * return a wrong D x).  The work is queued on cuda_stream (NULL: the legacy
 * default stream); no context is used.
 * Working memory is one fixed file-scope device array (11.9 MB, held by
 * every GPU that loads the library until the process exits) that stores the
 * rearranged links; each call rewrites the part it reads, so nothing needs
 * clearing, but calls that overlap on the GPU share it and race.  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first call on a device also loads the library's
 * device code there, so make it before any stream capture.
 * Errors: HP_EINVAL for a lattice above 20736 sites (12^4), ndim outside
 * [1, 4], nrhs < 1 or nrhs * V >= 2^31, host pointers or memory of another
 * device, an output that overlaps an input, a non-Wilson operator or
 * csw != 0 (the clover blocks would need workspace). */
hp_status hp_operator_apply_noalloc(const hp_operator* op, const hp_lattice* lat, int64_t nrhs,
                                    const double* in_dev, double* out_dev, void* cuda_stream);

/* Times `iters` launches of the Wilson stencil kernel in `precision` on
 * nrhs internal fields (CUDA events on the context stream) and reports the
 * mean time per launch and the algorithmic bytes / flops of one launch:
 * bytes = nrhs V (2 S + 4 L / nrhs) with S the bytes of one site's spinor
 * and L those of one link in that precision (each spinor read and written
 * once, the 4 links of a site read once for all right-hand sides),
 * flops = 1368 nrhs V.  All outputs are host scalars. */
hp_status hp_dslash_bench(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t precision,
                          int32_t nrhs, int32_t iters, double* ms_per_launch, double* bytes_per_launch,
                          double* flops_per_launch);

/* Per-kernel timing of everything the context launches while enabled
 * (CUDA events around each launch).  hp_profile_report writes a JSON
 * object {"kernel": {"launches": n, "ms": t}, ..., "_autotune": {key: choice}}
 * into buf (host, size bytes, NUL-terminated, truncated if short) and clears
 * the timing records. */
hp_status hp_profile_enable(hp_ctx* ctx, int32_t on);
/* Number of kernels the context has launched since its creation (kernels
 * replayed from captured graphs included), into *out (host). */
hp_status hp_launch_count(hp_ctx* ctx, int64_t* out);
hp_status hp_profile_report(hp_ctx* ctx, char* buf, int64_t size);

#ifdef __cplusplus
}
#endif

#endif /* HPROBE_H */
