/*
 * tmnd.h — C ABI of libtmnd.so: GB300 (sm_103a) kernels for the shifted
 * systems (Qhat^2 + sigma_i) x_i = b of the even-odd reduced, non-degenerate
 * twisted-mass Wilson operator (arXiv:1805.09584).
 *
 * Operator (Sec. 2, Eqs. "non-degenerate" and "Wilson" with c_sw = 0), in the
 * hopping-parameter normalisation (2 kappa times the paper's form, with
 * m + 4 = 1/(2 kappa)):
 *     D   = 1 - kappa H + 2 i kappa mu_bar (gamma_5 (x) tau_3) - 2 kappa eps_bar (1 (x) tau_1)
 *     H psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)
 *     Mhat = A - kappa^2 H_oe A^-1 H_eo          (even-odd Schur complement on odd sites, Sec. 2)
 *     A    = 1 + 2 i kappa mu_bar gamma_5 tau_3 - 2 kappa eps_bar tau_1
 *     Qhat = (gamma_5 (x) tau_1) Mhat,  Qhat^2 = Mhat^+ Mhat     (Eq. "g5tau1-hermiticity")
 * Gamma matrices: chiral basis, gamma_5 = diag(1,1,-1,-1) (Sec. 2);
 * gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i sigma_k],[i sigma_k,0]] in 2x2 blocks.
 * Lattice: dims = {T, X, Y, Z}, all even, mu = 0 is time; periodic in space,
 * antiperiodic in time when `antiperiodic_t` is set.  Site parity is
 * (t+x+y+z) & 1; the reduced system lives on the odd sites.
 *
 * Conventions for every entry point:
 *   - Device pointers are caller-owned (e.g. torch tensors' data_ptr()).  The
 *     library owns only the gauge handle, its packed links and a grow-only
 *     workspace inside the handle.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     stream-ordered and asynchronous unless stated otherwise.
 *   - Errors are returned as tmnd_status, never by aborting; a message is
 *     available from tmnd_last_error() (thread-local).  Invalid input is
 *     rejected with TMND_ERR_ARG before anything is launched.
 *   - A gauge handle may be used by one host thread at a time.
 *
 * Layouts
 *   canonical links (host) : complex128 [4][T][X][Y][Z][3][3], row-major, mu slowest.
 *   canonical spinor       : complex128 [nrhs][V/2][2 flavour][4 spin][3 colour]
 *                            on odd sites; odd half-index = lex >> 1 with
 *                            lex = ((t*X + x)*Y + y)*Z + z.
 *   internal spinor (TMND_F64): per right-hand side, 24 planes of V/2
 *                            complex128 values, plane c = flavour*12 + spin*3 + colour,
 *                            i.e. element (c, h) at offset (c * V/2 + h) complex
 *                            numbers; right-hand sides follow one another.
 *                            tmnd_spinor_bytes() gives the size of one.
 */
#ifndef TMND_H
#define TMND_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TMND_OK = 0,
    TMND_ERR_ARG = 1,      /* invalid argument (odd dims, sigma <= 0, bad pointer alignment, ...) */
    TMND_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    TMND_ERR_OOM = 3,      /* device allocation failed */
    TMND_ERR_NOCONV = 4,   /* solver reached maxiter before every required shift converged */
    TMND_ERR_NAN = 5,      /* NaN/Inf met in a reduction */
    TMND_ERR_TIMEOUT = 6,  /* a bounded wait gave up */
    TMND_ERR_NOTSU3 = 7    /* a link failed the SU(3) check at gauge creation */
} tmnd_status;

typedef enum {
    TMND_F64 = 0,          /* FP64 storage and arithmetic: 24 complex128 planes per RHS */
    TMND_F32 = 1,          /* FP32 storage: 24 complex64 planes per RHS */
    TMND_S16 = 2           /* 16-bit fixed-point storage with FP32 arithmetic, in blocks of
                              8 consecutive sites (800 bytes): 6 planes of 8 16-byte words
                              (word = one complex component, real part in the low 16 bits,
                              imaginary in the high 16 bits, component c = flavour*12 +
                              spin*3 + colour, plane c/4), then the 8 sites' scales
                              max|v|/32767 as floats; 100 bytes per site */
} tmnd_prec;

typedef enum {
    TMND_OP_MHAT = 0,      /* out = Mhat in                            (Sec. 2 even-odd reduction) */
    TMND_OP_MHAT_DAG = 1,  /* out = Mhat^+ in                          */
    TMND_OP_QHAT2 = 2,     /* out = (Mhat^+ Mhat + sigma) in           (Eq. "shifted_linear") */
    TMND_OP_QHAT = 3,      /* out = (gamma_5 (x) tau_1) Mhat in         (Eq. "g5tau1-hermiticity") */
    TMND_OP_S16 = 16,      /* flag OR-ed into the op: apply the sloppy operator (FP32 arithmetic,
                              16-bit links and intermediates) to TMND_S16 spinors */
    TMND_OP_F32 = 32       /* flag OR-ed into the op (TMND_OP_MHAT, _MHAT_DAG, _QHAT2): the FP32
                              operator (FP32 arithmetic, FP32 links and intermediates, relative
                              error ~1e-7) on TMND_F32 spinors */
} tmnd_op;

typedef struct {
    int dims[4];           /* {T, X, Y, Z}: each even and >= 2; V/2 < 2^31 */
    double kappa;          /* hopping parameter, m + 4 = 1/(2 kappa) */
    double mu_bar;         /* twisted mass mu_bar of Eq. "non-degenerate" */
    double eps_bar;        /* mass splitting eps_bar of Eq. "non-degenerate" */
    int antiperiodic_t;    /* 1: antiperiodic time boundary */
} tmnd_action;

typedef struct tmnd_gauge tmnd_gauge;

/* Create a gauge handle on the current CUDA device.  Copies `host_links`
 * (canonical layout, host memory, read only during the call) to the device
 * and packs it per parity and direction, in FP64 (18 reals per link) and in
 * 16-bit fixed point (rows 0 and 1, scale 32767; row 2 rebuilt in the
 * kernels) for the sloppy operator.  `prec` is TMND_F64 or TMND_S16 (both
 * copies are made either way).  Every link is checked on the host
 * to be SU(3) (|U U^+ - 1| and |det U - 1| below 1e-10); a failing link gives
 * TMND_ERR_NOTSU3.  Synchronous.  (Sec. 2: U_mu(x) in SU(3).) */
tmnd_status tmnd_gauge_create(const double *host_links, const tmnd_action *act, int prec,
                              tmnd_gauge **out);

/* Release the handle and all device memory it owns.  Synchronises the device. */
void tmnd_gauge_destroy(tmnd_gauge *g);

/* Bytes of one internal FP64 spinor (one right-hand side) for this handle. */
size_t tmnd_spinor_bytes(const tmnd_gauge *g);

/* Bytes of one internal spinor of precision `prec` (tmnd_prec). */
size_t tmnd_spinor_bytes_prec(const tmnd_gauge *g, int prec);

/* Convert nrhs internal spinors between precisions (F64 <-> S16, F32 -> S16,
 * F64 <-> F32; same precision copies).  Quantisation to S16 rounds every
 * component to the nearest multiple of (site max)/32767.  Buffers must not
 * overlap; device pointers, 16-byte aligned. */
tmnd_status tmnd_spinor_convert(const tmnd_gauge *g, void *dst, int dst_prec, const void *src, int src_prec,
                                int nrhs, void *stream);

/* canonical (device) -> internal (device), nrhs right-hand sides.  The two
 * buffers must not overlap.  Layouts as above. */
tmnd_status tmnd_spinor_pack(const tmnd_gauge *g, void *dev_internal, const void *dev_canonical,
                             int nrhs, void *stream);

/* internal (device) -> canonical (device). */
tmnd_status tmnd_spinor_unpack(const tmnd_gauge *g, void *dev_canonical, const void *dev_internal,
                               int nrhs, void *stream);

/* out = op(in) for nrhs internal spinors (see tmnd_op).  `sigma` is used by
 * TMND_OP_QHAT2 only.  With TMND_OP_S16 in `op`, in and out are TMND_S16
 * spinors and the operator is the sloppy one (FP32 arithmetic on 16-bit links,
 * intermediates rounded to 16 bits per site); then 1 <= nrhs <= 16 and every
 * stencil launch covers all nrhs right-hand sides (the links are read once per
 * launch and shared through the cache).  With TMND_OP_F32 in `op`, in and out
 * are TMND_F32 spinors and the operator is the FP32 one (one right-hand side
 * per launch sequence).  `out` and `in` must not overlap.  Uses
 * the handle's workspace (one even-site and one odd-site spinor per right-hand
 * side for TMND_OP_S16, one of each otherwise), growing it on first use.
 * (Sec. 2 even-odd Schur complement; Eq. "g5tau1-hermiticity".) */
tmnd_status tm_nd_apply(tmnd_gauge *g, void *out, const void *in, int op, double sigma,
                        int nrhs, void *stream);

/* No-allocation variant of tm_nd_apply.  The paper has no counterpart: this
 * is a library convenience.
 *
 * Same operation, arguments, layouts and stream semantics as tm_nd_apply, but
 * the two intermediate spinors (one even-site, one odd-site) live in one fixed
 * array of device memory declared inside the library instead of the handle's
 * workspace, so the call itself never allocates or frees device memory (no
 * cudaMalloc, no cudaFree, no allocating library routine).  It is meant for
 * callers that cannot allocate device memory at call time: programs whose
 * device memory is entirely owned by another allocator (a framework's caching
 * allocator, a fixed arena) with no room left for a library's own cudaMalloc,
 * and latency-critical loops that cannot accept the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.  (tm_nd_apply grows its workspace
 * with cudaMalloc the first time a handle needs it.)
 *
 *   - Limit: V/2 <= TMND_NOALLOC_MAX_VH odd sites (e.g. 16^4, 8^3x64);
 *     larger lattices are rejected with TMND_ERR_ARG.  The array takes
 *     2 x 24 x TMND_NOALLOC_MAX_VH complex128 = 24 MiB on every GPU that loads
 *     the library, until the process exits.
 *   - The current device must be the handle's device.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins.  The address is kept for the life of
 *     the process: after cudaDeviceReset (or any other teardown of the
 *     device's primary context) it is stale, so do not call this entry point
 *     again in a process that has reset the device.
 *   - Every call on a device (any handle, stream or host thread) uses the same
 *     array.  Calls whose executions overlap on the GPU race on it and give
 *     wrong results: order them (one stream, or events between streams).
 *   - The array keeps the last call's contents; everything a call reads from
 *     it is written earlier in the same call, so no clearing is needed. */
#define TMND_NOALLOC_MAX_VH 32768
tmnd_status tm_nd_apply_noalloc(const tmnd_gauge *g, void *out, const void *in, int op, double sigma,
                                int nrhs, void *stream);

/* Launch-shape autotuner of the sloppy (16-bit) stencil.  Its kernels run in
 * TMND_S16_SHAPES launch variants: 4 compiled shapes (threads per block x resident blocks
 * per SM the register budget is cut for x next-direction prefetch) x 4 loop orders (0: every
 * block walks its own chunk of sites, all right-hand sides of a site in turn; 1: the chunk
 * once per right-hand side; 2: all blocks sweep the lattice together by grid stride, all
 * right-hand sides of a site in turn; 3: grid stride over (group of 32 sites, right-hand
 * side) items, one per warp, a group's right-hand sides on consecutive warps);
 * tmnd_s16_shape_info.  For each lattice and number of right-hand sides per launch (1..16)
 * the library times every variant once on the current device, on scratch data, CUDA events,
 * best of 3 after a warm-up, for two sequences of 4 launches: (a) one 16-bit Qhat^2 + sigma
 * as tm_nd_apply runs it, and (b) one iteration of the sloppy multi-shift solver (the same
 * launches, the last one with the residual-update epilogue on FP32 residual planes); it keeps
 * the fastest variant of each for the rest of the process: (a) for tm_nd_apply, (b) for the
 * sloppy solves.  This happens on the first 16-bit tm_nd_apply or sloppy solve of that pair
 * (skipped while the stream is being captured: the default shape 0 is used then), or here,
 * ahead of time.  Synchronous; allocates its scratch for the call, 3 16-bit and 2 FP32
 * spinors per right-hand side (if that allocation fails, the default variant 0 is kept for
 * the pair and its times are reported as 0).
 *   shape_out : receives the chosen shape (may be NULL)
 *   ms_out    : TMND_S16_SHAPES doubles, each shape's time in ms (may be NULL)
 * tmnd_autotune reports sequence (a), tmnd_autotune_mms sequence (b); either call tunes both. */
#define TMND_S16_SHAPES 16
tmnd_status tmnd_autotune(tmnd_gauge *g, int nrhs, int *shape_out, double *ms_out, void *stream);
tmnd_status tmnd_autotune_mms(tmnd_gauge *g, int nrhs, int *shape_out, double *ms_out, void *stream);
/* Use shape `shape` for every later 16-bit stencil launch of this process (-1: back to the
 * tuned choice).  For tests and measurements; results do not depend on the shape. */
tmnd_status tmnd_s16_force_shape(int shape);
/* Threads per block, resident blocks per SM, prefetch flag (0/1) and loop order (0..3 as
 * above) of a variant (NULL outputs skipped). */
tmnd_status tmnd_s16_shape_info(int shape, int *threads, int *blocks_per_sm, int *prefetch, int *order);

#define TMND_MAX_SHIFTS 32

typedef struct {
    double rho;            /* stop shift i when its residual |r_i| <= rho |b| (Sec. 3.1 criterion) */
    int maxiter;           /* iteration cap; TMND_ERR_NOCONV if reached */
    int nsolve;            /* the first nsolve shifts must converge; the base system is
                              sigma[nsolve-1]; shifts after it are guess shifts (Sec. 4.2.2)
                              iterated along, never required to converge.  0 = all. */
    int check_every;       /* iterations between host convergence checks (0 = 32) */
    int profile;           /* 1: time the stencil and update kernels of every iteration with
                              CUDA events (filled into hop_ms / update_ms) */
    int prec;              /* TMND_F64 (0): plain FP64 multi-shift CG.
                              TMND_S16: mixed precision.  A sloppy multi-shift CG (FP32
                              arithmetic, 16-bit stencil vectors and links, FP32 residual,
                              FP64 dot-product accumulation) down to rho_inner, then FP64
                              defect correction per (RHS, shift) pair: FP64 true residual d;
                              an inner refinement in FP32 (batched sloppy CGs on the 16-bit
                              operator, each reducing its residual by the factor still needed
                              but at most max(rho_inner, 1e-4), each followed by the residual
                              of the accumulated correction with the FP32 operator, up to 4);
                              FP64 update; repeated until every required shift's FP64 true
                              residual is <= rho (one round is the rule). */
    double rho_inner;      /* TMND_S16: relative tolerance of the first sloppy multi-shift solve
                              (0 = 1e-5) */
    double *ab_hist;       /* optional host array: receives (alpha_k, beta_k), k = 1.., of the base
                              recursion of the first RHS (the Lanczos coefficients), zero-padded */
    int ab_hist_len;       /* length of ab_hist in doubles (2 per iteration) */
    int batch;             /* TMND_S16: right-hand sides the sloppy multi-shift solver iterates
                              together, every 16-bit stencil launch covering all of them
                              (0 = min(nrhs, 16); 1 = one at a time).  The FP64 defects are taken
                              one (RHS, shift) pair at a time; the inner refinements of up to
                              min(batch x nsolve, 16) pairs share each stencil launch. */
} tmnd_solve_params;

typedef struct {
    int iters;                             /* Krylov iterations of the base system */
    int conv_iter[TMND_MAX_SHIFTS];        /* iteration after which shift i froze, -1 if never */
    double true_res[TMND_MAX_SHIFTS];      /* |b - (Qhat^2 + sigma_i) x_i| / |b|, FP64, recomputed
                                              with the operator after the solve (max over RHS) */
    double zeta[TMND_MAX_SHIFTS];          /* final zeta_i of the recursion (last RHS) */
    double hop_ms;                         /* profile: device time of the 4 stencil launches per
                                              iteration, summed over iterations and RHS */
    double update_ms;                      /* profile: device time of the scalar + multi-shift
                                              update launches, summed likewise */
    long long launches;                    /* kernels this call launched (early-exit ones included) */
    int refine_rounds;                     /* TMND_S16: defect-correction rounds (max over RHS) */
    int refine_iters;                      /* TMND_S16: sloppy CG iterations of the corrections (sum) */
    int fp64_applies;                      /* FP64 applications of Qhat^2 + sigma (certification and
                                              defect correction, summed over RHS) */
    int f32_applies;                       /* TMND_S16: FP32 applications of Qhat^2 + sigma (the inner
                                              residuals of the defect correction) */
    double mms_ms;                         /* TMND_S16: wall time of the sloppy multi-shift solves */
    double fp64_ms;                        /* TMND_S16: wall time of the FP64 defects (true residuals) */
    double refine_ms;                      /* TMND_S16: wall time of the rest of the defect correction
                                              (sloppy corrections, FP32 residuals, FP64 updates) */
} tmnd_solve_info;

/* Multi-mass-shift CG (Sec. 1 "standard" solver; Sec. 4.2.2) for
 * (Qhat^2 + sigma_i) x_i = b, i < nshift, for each of nrhs right-hand sides.
 *   b      : device, nrhs internal spinors (read only)
 *   sigma  : host, nshift values, strictly descending, > 0 (descending order of Sec. 4.2.1)
 *   x      : host array of nshift device pointers; x[i] holds nrhs internal
 *            spinors and receives the solutions (overwritten, no initial guess)
 *   info   : may be NULL
 * Returns after the solve has finished (synchronous on `stream`).  Uses the
 * handle's workspace (4 + nshift spinors per right-hand side). */
tmnd_status mms_cg_solve(tmnd_gauge *g, const void *b, int nrhs, const double *sigma, int nshift,
                         void *const *x, const tmnd_solve_params *params, tmnd_solve_info *info,
                         void *stream);

/* Lagrange-interpolated initial guess (Sec. 4.2.1; App. B):
 *   out = sum_{j<k} l_j(target) xs[j],   l_j(m) = prod_{i != j} (m - m_i)/(m_j - m_i)
 * with the weights computed on the host in FP64 over `nodes` (host, k distinct
 * shifts, 1 <= k <= 8) and the combination done on the device.
 *   xs  : host array of k device pointers, each nrhs internal spinors
 *   out : device, nrhs internal spinors (may not alias any xs[j])
 *   lebesgue_out : host, may be NULL; receives gamma_k(target) = sum |l_j|. */
tmnd_status lagrange_guess(const tmnd_gauge *g, const double *nodes, const void *const *xs, int k,
                           double target, void *out, int nrhs, double *lebesgue_out, void *stream);

/* Lagrange weights l_j(target), j < k, over k distinct finite nodes (Sec. 4.2.1), and the
 * Lebesgue function gamma_k(target) = sum_j |l_j| (App. B; gamma may be NULL).  Host
 * function, FP64.  w: k doubles.  1 <= k <= 8. */
tmnd_status tmnd_lagrange_weights(const double *nodes, int k, double target, double *w, double *gamma);

/* Degree truncation of the Lagrange guess (App. B: where the Lebesgue function grows,
 * lower the degree of the interpolation to keep the residual bound rho gamma_k small).
 * Host function.  `nodes` lists k candidate shifts in order of preference (nearest to the
 * target first); *k_used receives the largest k' <= k such that the first k' nodes give
 * gamma_k'(target) <= gamma_max (k' >= 1: gamma_1 = 1), *gamma (may be NULL) that
 * gamma_k'(target).  1 <= k <= 8, distinct finite nodes, gamma_max >= 1, else TMND_ERR_ARG. */
tmnd_status tmnd_lagrange_degree(const double *nodes, int k, double target, double gamma_max, int *k_used,
                                 double *gamma);

/* Quadratic form of a guess residual (App. B): for solutions x_j of the shifts nodes[j]
 * with Gram matrix G (host, 2 k k doubles, row-major, re/im interleaved: G_jq = <x_j, x_q>),
 * H (host, k k doubles) = Re((target - s_j) G_jq (target - s_q)) / bb.  With exact x_j and
 * weights summing to 1, w^T H w = |b - (Qhat^2 + target) sum_j w_j x_j|^2 / bb, bb = |b|^2.
 * Host function.  1 <= k <= 8, bb > 0. */
tmnd_status tmnd_guess_quadratic_form(const double *G, const double *nodes, int k, double target, double bb,
                                      double *H);

/* ---------------------------------------------------------------- multigrid
 * Aggregation-based two-level multigrid (Sec. 3, DD-alphaAMG; Sec. 3.2 for the
 * doublet), FP32.  Layouts:
 *   fine MG vector   : full lattice, complex64 [parity][ncomp][V/2] per RHS
 *                      (ncomp = 12 for one flavour, 24 for the doublet; component
 *                      = flavour*12 + spin*3 + colour; parity 0 = even first)
 *   coarse vector    : complex64 [nrhs][nblock][2 flavour][2 chirality][nvec],
 *                      blocks in lexicographic order of their block coordinates
 *   prolongator P    : complex64 [nblock][2 chirality][nvec][block site][6], block site
 *                      s = ((it*bx + ix)*by + iy)*bz + iz, 6 = (spin within chirality)*3 + colour
 *   coarse operator  : complex64 [nblock][9][2 nvec][2 nvec], direction 0 = self,
 *                      1 + 2 mu + (0: neighbour block in +mu, 1: in -mu) */
typedef struct tmnd_mg tmnd_mg;

typedef struct {
    int block[4];              /* aggregate size {bt, bx, by, bz}; each divides dims */
    int nvec;                  /* test vectors per chirality, 1..32 (N_v of Sec. 3) */
    double coarse_mu_factor;   /* d of Sec. 3: coarse twisted mass d*mu_bar (<= 0: 1) */
    int coarse_simt;           /* 0: mg_coarse_apply on the tensor cores (tcgen05, TF32 operands,
                                  FP32 accumulation) whenever 2 nvec % 4 == 0 and nrhs <= 16,
                                  else FP32 CUDA cores; 1: always FP32 CUDA cores */
    double wait_limit_s;       /* every wait inside the tensor-core kernel gives up after this many
                                  seconds (0 = 2 s; at most 60); the kernel then ends with the
                                  handle's timeout flag set (see tmnd_mg_status) */
    int stall_test;            /* testing hook, 0 normally: the next stall_test tensor-core applies
                                  make their MMA warps wait on a barrier that nothing completes, so
                                  that the wait runs out after wait_limit_s and the error path
                                  (drain of copies and MMAs in flight, flag, clean exit) runs */
    int smoother;              /* 0: minimal-residual steps on the whole lattice; 1: SAP (Schwarz
                                  alternating procedure, the DD-alphaAMG smoother of Sec. 3) on the
                                  aggregation blocks (at most 256 sites each): per sweep and per
                                  colour of a red/black block colouring, the residual on the whole
                                  lattice, then sap_mr minimal-residual steps on every block of that
                                  colour with the block-local operator (hops leaving the block
                                  dropped), solved independently in parallel */
    int sap_mr;                /* SAP: minimal-residual steps per block solve (0 = 4) */
} tmnd_mg_params;

/* Build the hierarchy from `nvec` caller-provided test vectors (device, FP32
 * single-flavour fine MG vectors, one after another): orthonormalise them per
 * aggregate and chirality by Gram-Schmidt into a Gamma_5-compatible P (Sec. 3),
 * and assemble D_W,c = P^+ D_W P (Sec. 3) and G_odd = P^+ gamma_5 Pi_odd P (the
 * odd-site shift of the case-C systems).  Synchronous. */
tmnd_status tmnd_mg_create(tmnd_gauge *g, const tmnd_mg_params *p, const void *test_vectors, tmnd_mg **out);
void tmnd_mg_destroy(tmnd_mg *mg);

/* Bytes of one coarse doublet vector (one RHS). */
size_t tmnd_mg_coarse_bytes(const tmnd_mg *mg);

/* out_c = P_ND^+ in (restriction of nrhs fine doublet MG vectors), P_ND = P (x) 1_2 (Sec. 3.2). */
tmnd_status tmnd_mg_restrict(const tmnd_mg *mg, void *out_c, const void *in_fine, int nrhs, void *stream);

/* out = P_ND in_c (prolongation of nrhs coarse vectors). */
tmnd_status tmnd_mg_prolong(const tmnd_mg *mg, void *out_fine, const void *in_c, int nrhs, void *stream);

/* out_c = D'_c in_c for nrhs coarse doublet vectors, with the coarse doublet operator
 * (Sec. 3.2, Eq. "non-degenerate_coarse", hopping normalisation)
 *   D'_c = D_W,c (x) 1 + i 2 kappa d mu_bar (Gamma_5,c (x) tau_3) - 2 kappa eps_bar (1 (x) tau_1)
 *          + i odd_shift_s (tau_1 (x) G_odd)
 * (the last term is the coarse image of + i s gamma_5 tau_1 on odd sites, the shift
 * of the case-C systems).  9-point stencil over blocks.  Vectors 16-byte aligned.
 * Tensor cores (see tmnd_mg_params.coarse_simt): nrhs <= 16, 2 nvec % 4 == 0; the
 * dense blocks and the vectors enter the products as TF32 (relative error ~1e-3),
 * sums in FP32; a wait that gives up in the kernel is reported as TMND_ERR_TIMEOUT
 * by the next tmnd_mg_status / tmnd_mg_solve / tmnd_hybrid_solve.  The handle holds the operand
 * tiles of one application: one mg_coarse_apply at a time per handle.  CUDA cores:
 * nrhs * 4 nvec <= 1024, FP32 throughout. */
tmnd_status mg_coarse_apply(const tmnd_mg *mg, void *out_c, const void *in_c, int nrhs, double odd_shift_s,
                            void *stream);

/* Adaptive (bootstrap) setup (Sec. 3: the multigrid's own solves improve the test vectors
 * it is built from).  Every one of the nvec test vectors v (device, single-flavour fine MG
 * vectors as for tmnd_mg_create, updated in place) is replaced by the flavour-0 part of
 * w ~ D_ND^-1 (v, 0) from `iters` outer iterations of mg's two-level method (s = 0; MR/SAP
 * smoothing as configured, 2 steps), normalised; then a new hierarchy is built from the
 * improved vectors with parameters p and returned in *out (the caller destroys both
 * handles).  Call again on the result for more rounds.  Synchronous. */
tmnd_status tmnd_mg_bootstrap(tmnd_mg *mg, const tmnd_mg_params *p, void *test_vectors, int iters, tmnd_mg **out,
                              void *stream);

/* Waits for the device, then reports whether a tensor-core coarse apply on this handle gave
 * up a bounded wait since the last check: TMND_ERR_TIMEOUT (and the flag is cleared), else
 * TMND_OK.  The handle stays usable either way.  Synchronous. */
tmnd_status tmnd_mg_status(const tmnd_mg *mg);

/* out = D' in on the full lattice (fine doublet MG vectors, FP32), with
 *   D' = D_ND + i s (gamma_5 (x) tau_1) Pi_odd
 * (Eq. "non-degenerate" in the hopping normalisation; the odd-site term makes
 * the odd Schur complement Mhat + i s gamma_5 tau_1, the operator of the case-C
 * systems (Qhat + i s) y = b, Sec. 3.1 Eq. "lindif"). */
tmnd_status tmnd_dnd_full_apply(tmnd_gauge *g, void *out, const void *in, double s, void *stream);

/* Solve D' x = b (fine doublet MG vectors, FP32; x holds the initial guess and
 * receives the solution) by flexible GCR(restart) preconditioned with one
 * two-level V-cycle per iteration (Sec. 3, Eq. "error_propagation"): `nu`
 * pre- and post-smoothing steps (minimal residual on the whole lattice, or SAP sweeps,
 * per the handle's smoother) and a coarse GCR on mg_coarse_apply.  Stops at |b - D'x| <= tol |b| or after maxiter outer
 * iterations; iters / res (relative residual, FP32 operator) may be NULL.
 * Synchronous; allocates its scratch for the call. */
tmnd_status tmnd_mg_solve(tmnd_mg *mg, void *x, const void *b, double s, double tol, int maxiter, int restart,
                          int nu, int *iters, double *res, void *stream);

/* Relax nvec single-flavour fine MG vectors (device, in place) towards the
 * near-null space of D_TM(mu_bar): `iters` steps x <- x - w D x with
 * w = <Dx, x>/<Dx, Dx> (minimal residual on D x = 0), then normalise.  The
 * relaxed vectors are the test vectors of tmnd_mg_create (Sec. 3 setup). */
tmnd_status tmnd_mg_smooth_vectors(tmnd_gauge *g, void *vecs, int nvec, int iters, void *stream);

typedef struct {
    double rho;            /* target relative residual of every shift (FP64 true residual) */
    int maxiter;           /* iteration cap of the multi-shift and defect-correction solves */
    int prec;              /* TMND_F64 or TMND_S16 for the multi-shift part (see tmnd_solve_params) */
    double rho_inner;      /* sloppy tolerance (0 = 1e-5) */
    int n_guess;           /* shifts after the n_mms largest iterated along in the multi-shift
                              CG as guesses (Sec. 4.2.2; the paper uses 2) */
    int guess;             /* remaining shifts: 1 = Lagrange guess over the nearest <= 8 solved
                              shifts (Sec. 4.2.1), 0 = zero start, 2 = learned: weights from `net`
                              over the solutions of the 8 shifts just above (n_mms >= 8; the
                              network's features use the first RHS's base-recursion history) */
    double mg_tol;         /* relative tolerance of each case-C MG solve (0 = 1e-4; the solve is
                              FP32, the FP64 defect correction finishes the shift).  A shift whose
                              guess (RHS 0) already has an FP64 relative residual <= mg_tol skips
                              the multigrid for all its RHS */
    int mg_maxiter, mg_restart, mg_nu;   /* 0 = 100, 24, 4 (GCR(8) stagnates on the indefinite
                                            full-lattice operator at small shifts) */
    const struct tmnd_mlp *net;          /* guess = 2: a trained network (see tmnd_mlp_*), else NULL */
    double lebesgue_max;                 /* guess = 1: the nearest solved shifts (at most 8) are truncated to
                                            the longest nearest-first run whose Lebesgue function at the
                                            target is <= lebesgue_max (App. B; tmnd_lagrange_degree); 0 = 4 */
} tmnd_hybrid_params;

typedef struct {
    int mms_iters;                         /* base iterations of the multi-shift part */
    double guess_res[TMND_MAX_SHIFTS];     /* FP64 relative residual of each remaining shift's initial
                                              guess (RHS 0) */
    int mg_iters[TMND_MAX_SHIFTS];         /* outer MG iterations of the two case-C solves (RHS 0); the
                                              GCR stops at once when the guess already meets mg_tol */
    double true_res[TMND_MAX_SHIFTS];      /* final FP64 relative residuals (max over RHS) */
    int fp64_applies;                      /* FP64 operator applications */
    int refine_iters;                      /* sloppy defect-correction iterations */
    double shift_ms[TMND_MAX_SHIFTS];      /* wall time of each non-MMS shift's guesses, MG solves and
                                              batched defect correction (all RHS); the MMS part's in
                                              mms_ms */
    double mms_ms;                         /* wall time of the multi-shift part (all RHS) */
    int lag_nodes[TMND_MAX_SHIFTS];        /* guess = 1: interpolation nodes used for each shift */
    double lebesgue[TMND_MAX_SHIFTS];      /* guess = 1: gamma of those nodes at the shift */
    long long launches;                    /* kernels launched by the multi-shift part and the defect
                                              corrections (the multigrid's own launches not counted) */
    int f32_applies;                       /* FP32 applications of Qhat^2 + sigma (inner residuals) */
} tmnd_hybrid_info;

/* Hybrid solve of (Qhat^2 + sigma_i) x_i = b (Sec. 4.3): multi-shift CG for
 * the n_mms largest shifts, case-C multigrid solves from guesses for the rest
 * (see above), every shift finished by FP64 defect correction to hp->rho.
 * mg may be NULL: then the remaining shifts go from their guesses straight to the
 * defect correction (sloppy CG on the FP64 defect).  The remaining shifts are taken in
 * descending order; for each, every right-hand side gets its guess (and case-C solves),
 * then the defect corrections of all right-hand sides of that shift run as one batched
 * sloppy solve (up to 16 per stencil launch).
 * b, x as in mms_cg_solve (FP64 internal odd spinors).  Synchronous. */
tmnd_status tmnd_hybrid_solve(tmnd_gauge *g, tmnd_mg *mg, const void *b, int nrhs, const double *sigma, int nshift,
                              int n_mms, void *const *x, const tmnd_hybrid_params *hp, tmnd_hybrid_info *info,
                              void *stream);

/* Copy P, D_W,c and G_odd to host buffers (any may be NULL); for tests and inspection. */
tmnd_status tmnd_mg_export(const tmnd_mg *mg, void *P_host, void *Dc_host, void *Godd_host);

/* ------------------------------------------------------------ learned guess
 * Not in the paper; it extends the Lagrange guesses (Sec. 4.2.1).  A network
 * F -> 64 -> 64 -> 2 (tanh) predicts two log-poles o_k for a target shift sigma_t;
 * with p_k = exp(o_k) the weights over the solutions of 8 solved shifts sigma_j are
 *   w_j = l_j(sigma_t) prod_k (p_k + sigma_j) / (p_k + sigma_t)
 * (Lagrange interpolation of prod_k (p_k + sigma) x(sigma), divided back): they sum
 * to 1 for any poles (partition of unity, App. B) and tend to the Lagrange weights
 * as p_k -> infinity.
 * Parameters: FP32 [mu (F) isd (F) W1 (64xF) b1 W2 (64x64) b2 W3 (2x64) b3], row-major;
 * mu/isd standardise the inputs, x -> (x - mu) * isd, and are not trained.
 * Samples: X device float [N][F] (features); S device double [N][9] = (sigma_t,
 * sigma_1..sigma_8); H device double [N][8][8] row-major = Re(D G D), G = Gram matrix
 * of the 8 solutions / |b|^2, D = diag(sigma_t - sigma_j).  Loss per sample:
 * log(w^T H w + floor) -- with exact solutions and sum w = 1, w^T H w is the squared
 * relative residual of the guess; floor (>= 0, e.g. rho^2 of the solves that made the
 * data) stands for the residuals the solutions still carry.  Batch loss = mean. */
typedef struct tmnd_mlp tmnd_mlp;
int tmnd_mlp_num_params(int F);
/* Parameters initialised from `seed` (Gaussian, scale 1/sqrt(fan-in); last layer x0.1;
 * biases 0 except b3 = 3 (poles near 20: weights close to Lagrange's); mu = 0, isd = 1). */
tmnd_status tmnd_mlp_create(int F, unsigned long long seed, tmnd_mlp **out);
void tmnd_mlp_destroy(tmnd_mlp *m);
/* Copy the FP32 parameters to host_get and/or set them from host_set (either may be NULL). */
tmnd_status tmnd_mlp_params(tmnd_mlp *m, float *host_get, const float *host_set);
/* Set mu/isd to the per-feature mean and 1/standard deviation of X [N][F] (device; isd = 1
 * for a constant feature).  Call once on the training set before training. */
tmnd_status tmnd_mlp_fit_inputs(tmnd_mlp *m, const void *X, int N, void *stream);
/* Mean loss over N samples and its gradient (FP32 network, FP64 weights and loss);
 * grad_host: host float[num_params] or NULL (zero on mu/isd). */
tmnd_status tmnd_mlp_loss_grad(tmnd_mlp *m, const void *X, const void *S, const void *H, int N, double floor_q,
                               double *loss, float *grad_host, void *stream);
/* One Adam step (beta 0.9/0.999, eps 1e-8) on the mean loss of the N samples; loss may be NULL. */
tmnd_status tmnd_mlp_train_step(tmnd_mlp *m, const void *X, const void *S, const void *H, int N, double lr,
                                double floor_q, double *loss, void *stream);
/* Weights W (device double [N][8], rows sum to 1) from X and S, with BF16 layer weights
 * and FP32 accumulation; the weights themselves are formed in FP64. */
tmnd_status tmnd_mlp_predict(tmnd_mlp *m, const void *X, const void *S, int N, void *W, void *stream);
/* Network input (F = 20) for target shift `target` and 8 solved shifts `nodes`, from the
 * base recursion's (alpha_k, beta_k) history of niter iterations on the base shift sigma0
 * (host function; see mlp.cu for the feature list). */
tmnd_status tmnd_mlp_features(const double *nodes, double target, const double *ab_hist, int niter, double sigma0,
                              float *out);
/* G_jk = <x_j, x_k> (complex, FP64) of k <= 8 internal FP64 spinors (one RHS each);
 * G_host: 2*k*k doubles, row-major, interleaved re/im.  Synchronous. */
tmnd_status tmnd_gram(const tmnd_gauge *g, const void *const *xs, int k, double *G_host, void *stream);
/* out = sum_j w_j xs[j] for k <= 8 internal FP64 spinors with given FP64 weights (host). */
tmnd_status tmnd_lincomb(const tmnd_gauge *g, const double *w, const void *const *xs, int k, void *out, int nrhs,
                         void *stream);

/* ------------------------------------------- equivalent solutions (App. A, error and residual)
 * The study of App. A compares solutions of (Qhat^2 + mu^2) x = b that agree in exact
 * arithmetic: A, the direct solve; B, two consecutive solves with (Qhat +- i mu);
 * C, x_C = i/(2 mu) (x_+ - x_-) (Eq. "linear-combination"), with errors and residuals
 * against a known solution.  These two calls supply the complex combinations and the
 * local deviations; the solves are mms_cg_solve and tm_nd_apply (TMND_OP_QHAT).
 *
 * tmnd_lincomb_c: out = sum_j w_j xs[j] with complex weights, w = 2k doubles (re, im
 *   interleaved, host), k <= 8 internal FP64 spinors of nrhs right-hand sides each
 *   (device, 16-byte aligned); out may be one of the xs (element by element).
 *   Stream-ordered.  TMND_ERR_ARG for NULL, misaligned or non-finite arguments. */
tmnd_status tmnd_lincomb_c(const tmnd_gauge *g, const double *w, const void *const *xs, int k, void *out, int nrhs,
                           void *stream);
/* tmnd_site_norm_range: smallest and largest site norm |x(site)| (all 24 components of
 *   one odd site, FP64) over the nrhs internal FP64 spinors at x (device); min_max: 2
 *   doubles (host).  The "minimal and maximal local deviation" of App. A when x is an
 *   error vector.  Synchronous. */
tmnd_status tmnd_site_norm_range(const tmnd_gauge *g, const void *x, int nrhs, double *min_max, void *stream);

/* ------------------------------------------------------------ rational approximation
 * Zolotarev's optimal rational approximation of 1/sqrt(y) on eps < y < 1 (Sec. 4.1,
 * Eqs. "rational", "deviation", "zolotarev_shifts"):
 *   R(y) = a prod_{j=1..n} (y + c_{2j-1}) / (y + c_{2j}) = a (1 + sum_i q_i / (y + c_{2i}))
 * Host function.  c: 2n doubles (c_1 > c_2 > ... > c_2n > 0), q: n residues (Eq. "ratapp"),
 * *delta = max |1 - sqrt(y) R(y)| on (eps, 1) = d^2 / (1 + sqrt(1 - d^2))^2.
 * 1 <= n <= TMND_MAX_SHIFTS, 0 < eps < 1. */
tmnd_status tmnd_zolotarev(int n, double eps, double *a, double *c, double *q, double *delta);

/* out = R(Qhat^2 / lambda_max) b / sqrt(lambda_max) ~ (Qhat^2)^{-1/2} b (Sec. 4.1, Eq. "ratapp")
 * for a spectrum of Qhat^2 inside [lambda_min, lambda_max] (eps = lambda_min / lambda_max):
 * one mms_cg_solve of the n shifted systems (Qhat^2 + lambda_max c_{2i}) x_i = b with `params`
 * (nsolve 0: every shift converges) and one linear combination.  Per eigen-component the
 * relative error is at most delta (written to *delta_out, may be NULL) plus the solves'.
 * b, out: device, nrhs internal FP64 spinors.  Allocates n * nrhs spinors for the call.
 * Synchronous. */
tmnd_status tmnd_rational_apply(tmnd_gauge *g, const void *b, int nrhs, int n, double lambda_min,
                                double lambda_max, const tmnd_solve_params *params, void *out,
                                double *delta_out, tmnd_solve_info *info, void *stream);

/* ------------------------------------------------------------ hybrid cost model (Sec. 4.3)
 * Host functions.  Per shift s: t_CG(s) = a + b / ln(1 - 2/(sqrt(kappa(s)) + 1)),
 * kappa(s) = (lmax + s)/(lmin + s) (Eq. "CGtime2"); t_MG(s) = A + B / ln(1 - (C + s)/(L + s))
 * (Eq. "MGtime2"); the hybrid with the n largest of N descending shifts by multi-shift CG costs
 * c_HY(n) = t_CG(s_n) + sum_{i > n} t_MG(s_i) (Eq. "costwo").
 *   cg = {a, b, lmin, lmax}, mg = {A, B, C, L}; cost: N doubles (c_HY(1..N)); *n_opt = argmin. */
tmnd_status tmnd_hybrid_cost(const double *sigma, int N, const double *cg, const double *mg, double *cost,
                             int *n_opt);
/* Least-squares a, b of t_CG for measured times t[i] at shifts sigma[i] (N >= 2). */
tmnd_status tmnd_fit_cg_time(const double *sigma, const double *t, int N, double lmin, double lmax, double *a,
                             double *b);
/* A, B, C of t_MG: C on a log grid of `grid` points in (1e-8 L, 0.999 L), A and B by least
 * squares for each, the best residual kept (N >= 3). */
tmnd_status tmnd_fit_mg_time(const double *sigma, const double *t, int N, double L, int grid, double *A, double *B,
                             double *C);

/* Message for the last error on this host thread ("" if none). */
const char *tmnd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TMND_H */
