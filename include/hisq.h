/*
 * hisq.h -- C ABI of the GB300 (sm_103a) HISQ even/odd staggered operator library.
 *
 * The library applies the even/odd halves D_eo / D_oe of the HISQ staggered Dirac
 * operator and solves with A = M^dag M = 4 m^2 - D_eo D_oe by CG (plain FP64, mixed
 * precision with FP64 reliable updates, several right-hand sides) and multi-shift CG.
 * These are the operations the paper singles out: the Dslash stencil dominates the cost of
 * the CG, the CG takes about 60% of HISQ RHMC time, and the CG comes in multi-RHS,
 * multi-shift and mixed-precision forms (Sec. 3 and the module list of Sec. 2).
 *
 * Conventions (the paper writes no formula; these are the textbook HISQ ones):
 *   lattice    dims = {Lx, Ly, Lz, Lt}, each even and >= 4; periodic index wrap.
 *   site       idx = x + Lx*(y + Ly*(z + Lz*t)); parity = (x+y+z+t) mod 2, even = 0;
 *              cb = idx / 2 numbers the V/2 sites of one parity.
 *   operator   (D chi)(x) = sum_mu [ F_mu(x) chi(x+mu) - F_mu(x-mu)^dag chi(x-mu)
 *                                  + L_mu(x) chi(x+3mu) - L_mu(x-3mu)^dag chi(x-3mu) ]
 *              F = fat links, L = long (Naik) links with the Naik coefficient already
 *              included; staggered phases eta_mu(x) = (-1)^(x_0+..+x_{mu-1}) and the
 *              antiperiodic-t sign are folded in at load time (flags below). No factor
 *              1/2, so M = 2m + D and M^dag M on even sites is 4m^2 - D_eo D_oe.
 *              D_eo maps odd-site vectors to even sites; D_oe maps even to odd.
 *
 * Data at the boundary:
 *   links      host or device memory, complex128 interleaved (re, im),
 *              [t][z][y][x][mu][row][col], x fastest, mu = 0..3 = x, y, z, t (the layout
 *              hisq_smear writes, so smeared links can be loaded straight from the device).
 *   vectors    [rhs][cb][color] over the sites of one parity, complex numbers stored
 *              as (re, im) pairs of the precision's real type: HISQ_F64 and HISQ_DF64
 *              complex128, HISQ_F32 complex64, HISQ_F16 two IEEE binary16, HISQ_BF16 two
 *              bfloat16.
 *              Solver vectors are always complex128. A vector argument may point to
 *              device memory or to host memory (pageable or pinned); host data is
 *              staged through library-owned device buffers on the context's stream.
 *
 * Ownership and threading: the context owns its link storage and its device
 * workspaces; the caller owns every array it passes. One context serves one CUDA
 * stream; calls on one context must not run concurrently from several threads.
 * All work is issued on the context's stream; entry points that return results
 * to the host (solvers, host output vectors) synchronise that stream before they
 * return.
 *
 * Errors: every entry point returns HISQ_OK (0) or a negative HISQ_E* code and never
 * aborts, traps or prints. hisq_strerror() names a code; hisq_last_error() gives the
 * detail of the most recent failure in the calling thread.
 */
#ifndef HISQ_H
#define HISQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
  HISQ_OK = 0,
  HISQ_EINVAL = -1,      /* bad argument: dims, parity, null pointer, nrhs, precision not resident */
  HISQ_ENOLINKS = -2,    /* links not (fully) loaded */
  HISQ_ENOMEM = -3,      /* device or host allocation failed */
  HISQ_ECUDA = -4,       /* a CUDA runtime call failed; hisq_last_error() has its text */
  HISQ_ENONFINITE = -5,  /* NaN or Inf in links, source or an intermediate reduction */
  HISQ_ENOCONV = -6,     /* maxiter reached; x holds the last iterate, stats the true residual */
  HISQ_EBREAKDOWN = -7,  /* CG breakdown: <p, A p> <= 0 */
  HISQ_ETIMEOUT = -8     /* a bounded device-side wait ran out */
};

/* ---------------------------------------------------------------- precisions */
/*
 * HISQ_DF64 ("double-float") is an FP64-class precision that runs on the FP32 pipe: vectors
 * at the boundary are complex128 as for HISQ_F64, links are stored as pairs of FP32 words
 * (hi + lo, 16 bytes per complex entry like FP64) and the Dslash arithmetic is double-float
 * (error-free FP32 transformations, 2^-47 relative rounding per operation against FP64's
 * 2^-53). It exists because GB300 executes FP64 at ~1/60 of its FP32 rate, which makes the
 * FP64 Dslash arithmetic-bound; the double-float one is bandwidth-bound. Vector entries must
 * have magnitude below 2^127; entries below 2^-100 are treated as zero. The paper has no
 * counterpart. Not available for 16-bit link compression or the batched solver.
 */
typedef enum { HISQ_F64 = 0, HISQ_F32 = 1, HISQ_F16 = 2, HISQ_BF16 = 3, HISQ_DF64 = 4 } hisq_prec;
#define HISQ_PREC_BIT(p) (1u << (unsigned)(p))
#define HISQ_PREC_ALL 0x1Fu

/* ---------------------------------------------------------------- link-load flags */
#define HISQ_APPLY_PHASES 1u   /* multiply eta_mu(x) into fat and long links */
#define HISQ_ANTIPERIODIC_T 2u /* negate F_t at t = Lt-1 and L_t at t >= Lt-3 */

typedef struct hisq_ctx hisq_ctx;

/*
 * Create a context for one lattice (the gauge-field container of Sec. 2: one lattice, its links
 * and fields held in device memory). dims: {Lx, Ly, Lz, Lt}, each even and >= 4.
 * prec_mask: OR of HISQ_PREC_BIT(p) for every storage precision whose links should
 * be kept resident (HISQ_F64 is always added: reliable updates and true residuals
 * need it). stream: a cudaStream_t (NULL = legacy default stream), borrowed.
 * Allocates the link storage: 8 links x 18 reals x V per resident precision.
 * Errors: HISQ_EINVAL, HISQ_ENOMEM, HISQ_ECUDA.
 */
int hisq_create(hisq_ctx** out, const int dims[4], unsigned prec_mask, void* stream);

/* Free every device and host resource of the context. NULL is accepted. */
int hisq_destroy(hisq_ctx* ctx);

/*
 * Load fat and long links for the whole lattice (the link storage of Sec. 2 and Sec. 3: the HISQ
 * operator's smeared one-hop and Naik three-hop links, held in the precision each Dslash reads;
 * host or device arrays in the link layout above, V*4*9 complex128 each). flags: HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T.
 * The links are folded (phases, boundary sign) and converted to every resident
 * precision on the device; the input arrays are not kept. Returns HISQ_ENONFINITE if
 * any entry is NaN or Inf (the previous links are then no longer valid).
 */
int hisq_load_links(hisq_ctx* ctx, const double* fat, const double* lng, unsigned flags);

/*
 * Load the links of the t-slices [t_begin, t_begin + t_count) only; fat and lng then
 * hold t_count*Lz*Ly*Lx*4*9 complex128 each. Lets lattices whose host link arrays would
 * not fit in host memory be loaded slab by slab. The context is ready once every
 * t-slice has been loaded (with the same flags).
 */
int hisq_load_links_slab(hisq_ctx* ctx, int t_begin, int t_count, const double* fat, const double* lng,
                         unsigned flags);

/*
 * Long-link compression (the paper's "gauge field compression": store part of each link and
 * recompute the rest from its SU(3)/U(3) structure, Sec. 3). With naik != 0 the context also keeps
 * the first two rows of every folded long link in its FP32/FP16/BF16 storage, and those Dslash
 * applications read 12 reals per long link instead of 18 (16% fewer bytes per site), rebuilding
 * row 2 = conj(row0 x row1) / c with c = naik * eta_mu(x) * (antiperiodic sign), computed from
 * the site's coordinates. Requires every long link to be naik * SU(3) (as for long links made of
 * products of SU(3) links); hisq_load_links then returns HISQ_EINVAL otherwise. Call before loading
 * links (it invalidates loaded links); naik = 0 turns compression off. FP64 is never compressed.
 */
int hisq_set_long_compression(hisq_ctx* ctx, double naik);

/*
 * The Dslash stencil whose cost dominates the CG and which is bound by memory bandwidth (Sec. 3);
 * with nrhs > 1 one read of the links serves every vector, the multi-RHS form of Sec. 3.
 * out = D_eo in (out_parity = 0: out on even sites, in on odd sites), or
 * out = D_oe in (out_parity = 1). Vectors in precision prec (its links must be
 * resident), nrhs vectors of V/2 sites back to back; out and in must not overlap.
 * Arithmetic: FP64 for HISQ_F64, double-float for HISQ_DF64, FP32 for the others (16-bit
 * types are storage only). Asynchronous on the context's stream for device pointers.
 * Errors: HISQ_EINVAL (parity, nrhs < 1 or > 64, precision not resident), HISQ_ENOLINKS.
 */
int hisq_dslash(hisq_ctx* ctx, int out_parity, void* out, const void* in, int prec, int nrhs);

/*
 * out = (4 m^2 + sigma) in - D_eo D_oe in on even sites: the even-site operator M^dag M that the
 * CG of Sec. 2 and Sec. 3 inverts (two Dslash applications per CG iteration), shifted by sigma as
 * the multi-shift CG needs it. Same vector conventions as hisq_dslash. Errors as hisq_dslash, and
 * HISQ_EINVAL for mass < 0 or sigma < 0.
 */
int hisq_apply_A(hisq_ctx* ctx, void* out, const void* in, double mass, double sigma, int prec, int nrhs);

/*
 * The same two operators on the rhs-interleaved vector layout [cb][color][rhs]: the nrhs vectors of
 * one site are one contiguous block of 3 rows (colours) of nrhs complex numbers (out, in: V/2 such
 * blocks). This is the multi-RHS form of Sec. 3 laid out for the stencil: each of the 16 hops reads a
 * neighbour's vectors as one block with 16-byte loads, and one launch applies every link to all nrhs
 * vectors.
 * nrhs: 1..64, a multiple of 2 for HISQ_F32 and of 4 for HISQ_F16 / HISQ_BF16 (any for HISQ_F64 and
 * HISQ_DF64). Arithmetic, staging of host vectors and errors as hisq_dslash / hisq_apply_A
 * (HISQ_EINVAL also for an nrhs that is not such a multiple). The launch form (vectors per thread)
 * and block size are chosen by the autotuner at the first call per (precision, nrhs).
 * With 16-bit storage, 16 to 64 vectors and hisq_dslash_interleaved there are two forms: FP32 FMAs
 * on the CUDA cores, and the fifth-generation tensor cores (tcgen05.mma, one 64 x 8 x 128 product
 * per site, FP32 accumulation in TMEM). With the autotuner on, the first call per (precision,
 * nrhs) runs and times both (the output is written twice, with equal results up to rounding
 * order) and keeps the faster; hisq_tune_report lists the choice as
 * "dslash_path_il/l<prec>/n<nrhs> -> 1 (CUDA cores) or 2 (tensor cores)". A bounded tensor-core
 * wait that ran out is reported by that first call (HISQ_ECUDA is not raised; the form is then
 * not chosen) and writes NaN into the affected outputs.
 */
int hisq_dslash_interleaved(hisq_ctx* ctx, int out_parity, void* out, const void* in, int prec, int nrhs);
int hisq_apply_A_interleaved(hisq_ctx* ctx, void* out, const void* in, double mass, double sigma, int prec,
                             int nrhs);

/* ---------------------------------------------------------------- solvers */
typedef struct {
  int inner_prec;       /* HISQ_F64: plain FP64 CG. HISQ_DF64: plain CG with the double-float
                           operator (FP64 vectors and BLAS). HISQ_F32 / F16 / BF16: mixed
                           precision -- inner CG with links in that precision, spinors stored as
                           spinor_prec says, FP32 arithmetic, FP64 reductions and FP64 solution
                           accumulator, reliable updates in reliable_prec */
  int reliable_period;  /* inner iterations between reliable updates (default 50) */
  int use_graph;        /* 1: capture blocks of iterations in a CUDA graph (default 1) */
  int poll_every;       /* iterations between host convergence polls (default 25) */
  int reliable_prec;    /* operator precision of reliable updates and true residuals:
                           HISQ_F64 (default) or HISQ_DF64 (its links must be resident) */
  int vector_layout;    /* inner vectors of a mixed-precision solve with an even number of rhs:
                           0 (default) [rhs][cb][color], 1 interleaved per site ([cb][color][rhs],
                           read by the interleaved multi-RHS Dslash). Results agree up to rounding
                           order; the caller's x and b keep the boundary layout either way. On
                           GB300 the default is the faster at every rhs count measured */
  int spinor_prec;      /* storage of the inner vectors (r, p, Ap and the Dslash intermediate) of a
                           mixed-precision hisq_cg: HISQ_F32 (default), or 16-bit storage equal to
                           inner_prec (HISQ_F16 with FP16 links, HISQ_BF16 with BF16 links) with
                           vector_layout 0; arithmetic stays FP32, reductions and the solution FP64.
                           Other values, and 16-bit storage in hisq_multishift_cg, give HISQ_EINVAL */
} hisq_solver_opts;

typedef struct {
  int iters;                  /* CG iterations (inner iterations for mixed precision) */
  int reliable_updates;       /* FP64 residual recomputations */
  int converged;              /* 1 if every rhs / shift met its tolerance */
  double true_rel_residual;   /* max over rhs / shifts of ||b - (A+sigma) x|| / ||b||, FP64, at exit */
  double seconds;             /* wall time of the solve inside the library */
  double dslash_bytes;        /* algorithmic bytes of all Dslash applications in the solve */
  long long dslash_calls;     /* Dslash applications (one rhs-block counts once) */
  int shift_iters[64];        /* multi-shift: iteration at which each shift converged */
  double shift_residual[64];  /* true residual of each shift (multi-shift) or rhs (CG) */
  long long kernel_launches;  /* CUDA kernels this call executed (graph nodes included) */
  /* hisq_cg: estimates of the extreme eigenvalues of the solved operator (A + sigma of rhs 0) from
     the Lanczos tridiagonal matrix of rhs 0's CG coefficients (hisq_lanczos_extremes), over its
     longest run of iterations without a restart of the search direction; their ratio estimates the
     condition number. lanczos_steps = coefficients recorded (restart marks included). 0 if none. */
  double lambda_min, lambda_max;
  int lanczos_steps;
} hisq_solver_stats;

/*
 * Extreme eigenvalues of the Lanczos tridiagonal matrix that n CG coefficients define (alpha_k, beta_k
 * of iteration k: x += alpha_k p, p = r + beta_k p): T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1},
 * T_k,k+1 = sqrt(beta_k)/alpha_k, over the longest run of entries with alpha > 0 (alpha = 0 marks a
 * restart). They bound A's extreme eigenvalues from inside and converge to them as CG converges
 * (the Lanczos connection of CG, textbook; the paper has none). Host only; bisection on Sturm counts
 * to ~1e-15 relative. Errors: HISQ_EINVAL (null pointer, n < 1, no positive alpha).
 */
int hisq_lanczos_extremes(const double* alpha, const double* beta, int n, double* lmin, double* lmax);

/* Fill opts with the defaults above (inner_prec = HISQ_F64). */
void hisq_solver_opts_default(hisq_solver_opts* opts);

/*
 * The CG of Sec. 2 (module list: CG with multi-RHS and mixed-precision variants) and Sec. 3 (the
 * CG that takes about 60% of RHMC time), on the even-site operator A.
 * Solve A x_r = b_r (A = 4 m^2 - D_eo D_oe) for nrhs right-hand sides at once, each to
 * ||b_r - A x_r|| <= rel_tol ||b_r||, judged by the true FP64 residual at exit.
 * x: complex128 [nrhs][V/2][3], the initial guess on entry (zero is fine) and the
 * solution on exit; b: the sources, same layout. Host or device pointers.
 * opts may be NULL (defaults); stats may be NULL.
 * Errors: HISQ_EINVAL (mass <= 0, rel_tol <= 0, nrhs out of range, inner precision not
 * resident), HISQ_ENOLINKS, HISQ_ENONFINITE, HISQ_ENOCONV, HISQ_EBREAKDOWN, HISQ_ECUDA.
 */
int hisq_cg(hisq_ctx* ctx, double* x, const double* b, int nrhs, double mass, double rel_tol, int maxiter,
            const hisq_solver_opts* opts, hisq_solver_stats* stats);

/*
 * Multi-shift CG: (A + sigma_k) x_k = b for nshift shifts sigma_k >= 0 from one Krylov
 * space (the RHMC use of the CG, Sec. 2 and Sec. 3). x: nshift complex128 vectors
 * [nshift][V/2][3] (output; initial contents ignored); b: one source. rel_tol: nshift
 * tolerances. With opts->inner_prec != HISQ_F64 the shared Krylov space is built in
 * that precision (FP64 reductions and accumulators) and each shift is then refined
 * by mixed-precision CG with FP64 reliable updates until its true residual meets
 * its tolerance. nshift <= 64.
 */
int hisq_multishift_cg(hisq_ctx* ctx, double* x, const double* b, int nshift, const double* shifts,
                       double mass, const double* rel_tol, int maxiter, const hisq_solver_opts* opts,
                       hisq_solver_stats* stats);

/* ---------------------------------------------------------------- batches of lattices */
/*
 * A batch of independent lattices of (possibly) different sizes, solved together: every
 * step of the batched CG is one persistent launch over a tile table that covers all
 * lattices, and one CUDA graph holds a whole reliable cycle (inner iterations, fold, FP64
 * residual, reliable update). This is the many-small-lattices form of the paper's CG
 * (Sec. 2, Sec. 3); the paper itself batches right-hand sides, not lattices.
 * dims: nlat x 4 extents (each even and >= 4), nlat <= 256. FP64 and FP32 links are always
 * resident. Vectors of the batch: the even-site vectors of all lattices back to back,
 * complex128 [lattice][V_l/2][3]; hisq_batch_vector_offset gives lattice l's first complex
 * entry (l = nlat gives the total).
 */
typedef struct hisq_batch hisq_batch;
int hisq_batch_create(hisq_batch** out, int nlat, const int* dims, unsigned prec_mask, void* stream);
int hisq_batch_destroy(hisq_batch* batch);
/* Links of one lattice of the batch, as hisq_load_links. */
int hisq_batch_load_links(hisq_batch* batch, int lattice, const double* fat, const double* lng, unsigned flags);
long long hisq_batch_vector_offset(const hisq_batch* batch, int lattice);
long long hisq_batch_launch_count(const hisq_batch* batch);
/*
 * Solve A_l x_l = b_l (A_l = 4 m_l^2 - D_eo D_oe on lattice l) for every lattice to
 * ||b_l - A_l x_l|| <= rel_tol ||b_l||, verified in FP64. mass: nlat masses. opts->inner_prec
 * HISQ_F32 (mixed precision, FP64 reliable updates every reliable_period iterations) or
 * HISQ_F64. x: initial guess in, solution out; host or device. iters, true_res: optional
 * per-lattice outputs [nlat]. stats: aggregate (iters = the largest per-lattice count).
 */
int hisq_batch_cg(hisq_batch* batch, double* x, const double* b, const double* mass, double rel_tol, int maxiter,
                  const hisq_solver_opts* opts, hisq_solver_stats* stats, int* iters, double* true_res);

/* ---------------------------------------------------------------- learned preconditioner */
/*
 * A gauge-equivariant parallel-transport convolution (PTC) network used as the
 * preconditioner of a flexible CG (the project's extension of the paper's CG; the paper
 * has none). Layer: psi'_a(x) = sum_b sum_h W[a][b][h] (T_h psi_b)(x) over 9 hops
 * h = 0, +x, +y, +z, +t, -x, -y, -z, -t, with T_+mu psi(x) = F_mu(x) psi(x+mu) and
 * T_-mu psi(x) = F_mu(x-mu)^dag psi(x-mu) through the context's folded FP32 fat links.
 * Network: 1 -> channels -> 1 (channels = 8), linear; input an even-site vector embedded
 * with zeros on odd sites, output restricted to even sites. Channel mixing runs on the
 * tensor cores in BF16 with FP32 accumulation; master weights are FP32.
 * Weights: w1 [channels][1][9], w2 [1][channels][9], complex as (re, im) float pairs.
 * Network vectors: device, complex64 [nvec][V/2][3] (even sites).
 */
typedef struct hisq_ptc hisq_ptc;
int hisq_ptc_create(hisq_ptc** out, hisq_ctx* ctx, int channels);
/* Frees the network's buffers only; valid before or after its context is destroyed. */
int hisq_ptc_destroy(hisq_ptc* ptc);
/* Host or device FP32 weights in; resets the Adam moments. */
int hisq_ptc_set_weights(hisq_ptc* ptc, const float* w1, const float* w2);
int hisq_ptc_get_weights(hisq_ptc* ptc, float* w1, float* w2);
/* tied = 1: layer 2 becomes the adjoint of layer 1 (W2[0][a][h] = conj(W1[a][0][adj h]), adj
 * swapping +mu and -mu), so N = B^dag B is Hermitian positive semi-definite -- the form a CG
 * preconditioner wants. Training then updates w1 only, with the layer-2 gradient carried back;
 * g1 of hisq_ptc_train_step is the combined gradient. */
int hisq_ptc_set_tied(hisq_ptc* ptc, int tied);
/* Rebind the network (weights and Adam moments kept) to another context of the same lattice
 * shape, e.g. to train on several gauge fields. */
int hisq_ptc_bind(hisq_ptc* ptc, hisq_ctx* ctx);
/* z = N(r) for nvec even-site FP32 vectors (device), applied in the composed form of the linear
 * network (one odd-site and one even-site stencil pass on CUDA cores, weights rounded to BF16 as in
 * training). Asynchronous on the context's stream, like hisq_dslash. */
int hisq_ptc_apply(hisq_ptc* ptc, float* z, const float* r, int nvec);
/*
 * Loss = mean over npairs of |N(b_i) - x_i|^2 / |x_i|^2 and its gradients with respect to
 * conj(w1), conj(w2) (loss, g1, g2: optional host outputs); with lr > 0 one Adam step on the
 * FP32 master weights follows. b, x: device complex64 [npairs][V/2][3].
 */
int hisq_ptc_train_step(hisq_ptc* ptc, const float* b, const float* x, int npairs, float lr, float* loss, float* g1,
                        float* g2);
/*
 * Flexible CG (truncated to one previous direction, Notay 2000) preconditioned by the network:
 * z = N(r); p = z - (<q_old, z>/<q_old, p_old>) p_old; alpha = <p, r>/<p, A p> (complex in
 * general). Inner vectors FP32 with FP32 links, FP64 reductions and solution, FP64 reliable
 * update (true residual, restart p = N(r)) every opts->reliable_period iterations. Same
 * conventions and errors as hisq_cg (single rhs).
 */
int hisq_fcg(hisq_ctx* ctx, hisq_ptc* ptc, double* x, const double* b, double mass, double rel_tol, int maxiter,
             const hisq_solver_opts* opts, hisq_solver_stats* stats);

/* ---------------------------------------------------------------- no-allocation variant */
/*
 * Bytes of the fixed device scratch array behind hisq_apply_A_noalloc (32 MiB). Every GPU that
 * loads the library holds this array until the process exits.
 */
#define HISQ_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * hisq_apply_A_noalloc -- the paper has no counterpart; this is a service of the library.
 * Same result as hisq_apply_A, out = (4 m^2 + sigma) in - D_eo D_oe in, for callers that cannot
 * allocate device memory when they make the call: code whose device memory is owned by an
 * allocator that forbids foreign allocations, and latency-critical loops that cannot take the
 * device synchronisation of cudaMalloc. hisq_apply_A allocates its odd-site intermediate on first
 * use; this variant keeps it in a fixed file-scope device array of HISQ_NOALLOC_SCRATCH_BYTES and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 * in, out: device pointers only (host vectors would need staging buffers); nrhs * V/2 * 6 *
 * sizeof(real of prec) must not exceed HISQ_NOALLOC_SCRATCH_BYTES, else HISQ_EINVAL.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, once per
 * device, with that device current). The device
 * current at the call must be the one that was current at hisq_create, else HISQ_EINVAL.
 * All calls share the array: calls whose work overlaps on the GPU (several streams or host
 * threads at once) race on it. Nothing in it needs clearing: each call overwrites what it reads.
 */
int hisq_apply_A_noalloc(hisq_ctx* ctx, void* out, const void* in, double mass, double sigma, int prec, int nrhs);

/*
 * Rational function of A applied to a vector, as RHMC uses the multi-shift CG (Sec. 2: RHMC for
 * HISQ fermions; Sec. 3: multi-shift CG): out = a0 b + sum_k coeffs[k] (A + shifts[k])^-1 b, each
 * shifted system solved to rel_tol[k] by hisq_multishift_cg (same options). The coefficients of a
 * rational approximation are the caller's (the paper gives none). out, b: complex128 [V/2][3],
 * host or device. stats: those of the multi-shift solve.
 */
int hisq_rational_apply(hisq_ctx* ctx, double* out, const double* b, double a0, int nshift, const double* shifts,
                        const double* coeffs, double mass, const double* rel_tol, int maxiter,
                        const hisq_solver_opts* opts, hisq_solver_stats* stats);

/* ---------------------------------------------------------------- link smearing */
/*
 * Path coefficients of one smearing level of HISQ type (the HISQ action of the paper's simulations,
 * Sec. 1, builds its fat and long links this way; the coefficients are not in the paper and are the
 * caller's). For every site x and direction mu, with paths read as products of the links walked
 * (U_d(y) for a step +d from y, U_d(y-d)^dag for a step -d):
 *   fat_mu(x)  = one_link U_mu(x)
 *              + three_staple * sum of the  6 paths (nu, mu, -nu)                 nu != mu, both signs
 *              + five_staple  * sum of the 24 paths (rho, nu, mu, -nu, -rho)      nu, rho, mu distinct
 *              + seven_staple * sum of the 48 paths (sig, rho, nu, mu, -nu, -rho, -sig)  all distinct
 *              + lepage       * sum of the  6 paths (nu, nu, mu, -nu, -nu)
 *   long_mu(x) = naik U_mu(x) U_mu(x+mu) U_mu(x+2mu)
 * The staggered phases and the boundary sign are not applied (hisq_load_links folds them in).
 */
typedef struct {
  double one_link, three_staple, five_staple, seven_staple, lepage, naik;
} hisq_smear_coeffs;

/*
 * One smearing level on the device. thin: input links; fat, lng: outputs; all three device
 * pointers (16-byte aligned) in the link layout of hisq_load_links (V*4*9 complex128, so the
 * outputs can be passed to hisq_load_links directly). lng may be NULL (long links not formed).
 * Outputs must not overlap the input or each other. prec: the arithmetic, HISQ_F64 (IEEE FP64) or
 * HISQ_DF64 (double-float on the FP32 pipe, ~2^-47 relative rounding per operation); inputs and
 * outputs are binary64 either way. Uses 144 * 16 bytes of context workspace per site. Stream-ordered,
 * no host synchronisation. Errors: HISQ_EINVAL (null or host pointer, misaligned, overlapping,
 * non-finite coefficient, other prec), HISQ_ENOMEM, HISQ_ECUDA.
 */
int hisq_smear(hisq_ctx* ctx, double* fat, double* lng, const double* thin, const hisq_smear_coeffs* c, int prec);

/*
 * Projection of every link onto U(3): out = W (W^dag W)^{-1/2} for each 3x3 link W of in (device
 * pointers, link layout; out == in is allowed, partial overlap is not). FP64. Synchronises the
 * stream. Returns HISQ_EINVAL if some W^dag W is not positive definite (that link is copied
 * unchanged).
 */
int hisq_project_u3(hisq_ctx* ctx, double* out, const double* in);

/*
 * The two levels of the HISQ construction: W = project_u3(level-1 fat links of thin), then the
 * level-2 fat links of W into fat and the Naik product of W into lng (level1's naik is unused).
 * Arguments and errors as hisq_smear and hisq_project_u3 (synchronises the stream); also uses
 * V*4*9 complex128 of workspace for W.
 */
int hisq_hisq_links(hisq_ctx* ctx, double* fat, double* lng, const double* thin, const hisq_smear_coeffs* level1,
                    const hisq_smear_coeffs* level2, int prec);

/*
 * Free the context's device workspaces (staging buffers, solver and smearing scratch) and the solver
 * graphs cached on them; both are allocated again on demand by the next call that needs them.
 * Synchronises the stream first. Link storage and the autotuner's cache are kept. Errors:
 * HISQ_EINVAL (null context), HISQ_ECUDA.
 */
int hisq_release_workspaces(hisq_ctx* ctx);

/* ---------------------------------------------------------------- diagnostics */
const char* hisq_strerror(int code);
const char* hisq_last_error(void);

/* Algorithmic bytes of one Dslash application on one parity in precision prec with
 * nrhs vectors: (V/2) * (16 links * 18 + nrhs * (6 in + 6 out)) reals. */
double hisq_dslash_bytes(const hisq_ctx* ctx, int prec, int nrhs);

/* Number of CUDA kernels this context has executed so far (eager launches, autotuning
 * trials and every node of every graph launch). */
long long hisq_launch_count(const hisq_ctx* ctx);

/* Autotuner: choose launch shapes by timing (default on). The cache lives in the
 * context; hisq_tune_report writes one "key LxxLyxLzxLt -> choice" line per tuned kernel to buf
 * (choice = launch-form index * 10000 + block size). hisq_tune_load reads such a report back
 * into a context of the same lattice dims (lines for other dims are skipped), so a later run can
 * skip the timing launches; *loaded (may be NULL) receives the number of entries taken.
 * Errors: HISQ_EINVAL (null context or text, malformed line). */
int hisq_set_autotune(hisq_ctx* ctx, int enable);
int hisq_tune_report(const hisq_ctx* ctx, char* buf, size_t len);
int hisq_tune_load(hisq_ctx* ctx, const char* report, int* loaded);

/* Programmatic dependent launch (default on): each single-layout Dslash launch that a call makes on
 * the context's stream (hisq_dslash, hisq_apply_A and their variants, and the eager launches of the
 * solvers), and the two passes of hisq_ptc_apply, may be scheduled onto the GPU while the launch
 * before it in the stream drains, and wait on the device for that launch's results before they read
 * or write anything; results are unchanged. The CUDA graphs the solvers capture keep plain launches.
 * enable = 0 makes every launch a plain stream-ordered one. Errors: HISQ_EINVAL (null context). */
int hisq_set_pdl(hisq_ctx* ctx, int enable);

/*
 * Self-test of the failure path of the bounded device-side waits (the completion waits of the
 * tensor-core kernels and the grid-barrier wait of the fused CG update give up after a bounded
 * number of polls, flag the failure and return instead of hanging): launches one block that waits
 * on an mbarrier nothing arrives at and one that waits at a grid barrier whose generation nothing
 * advances. Returns HISQ_ETIMEOUT when both waits gave up as intended -- the expected result --
 * after which the context remains usable. The paper has no counterpart.
 */
int hisq_selftest_bounded_wait(hisq_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HISQ_H */
