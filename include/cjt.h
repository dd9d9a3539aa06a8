/*
 * cjt.h -- C ABI of the GB300 (sm_103a) Chebyshev--Jacobi transform library.
 *
 * The library computes, on one GPU, the forward and inverse Chebyshev--Jacobi
 * transforms of R. M. Slevinsky, "On the use of Hahn's asymptotic formula and
 * stabilized recurrence for a fast, simple, and stable Chebyshev--Jacobi
 * transform" (arXiv:1602.02618):
 *
 *   forward  c_cheb = T_N^{-1} P_N^{(alpha,beta)} c_jac        (Eq. "CJT", Sec. 1)
 *   inverse  c_jac  = P_N^{(alpha,beta)}^{-1} T_N c_cheb       (Eq. "iCJT", Sec. 1)
 *
 * where [P_N]_{j,n} = P_n^{(alpha,beta)}(x_j) and [T_N]_{j,k} = T_k(x_j) at the
 * N+1 Chebyshev--Lobatto points x_j = cos(pi j/N), j = 0..N.  The forward map
 * evaluates the Jacobi expansion at the Lobatto points by the paper's
 * partition (Sec. 2.2): Hahn's interior asymptotic formula as a sum of
 * diagonally scaled DCT-I/DST-I (Eq. "PNASY") inside the boxes, the
 * Clenshaw--Smith recurrence (Reinsch-modified near x = +-1, Sec. 4.2)
 * elsewhere, and finishes with the inverse scaled DCT-I.  The inverse map is
 * the transposed formula on the 2N grid with Clenshaw--Curtis weights
 * (Eq. "CJTT", Sec. 3.2).
 *
 * Conventions shared by every entry point:
 *  - All coefficient vectors are contiguous IEEE double arrays of length N+1
 *    (index n = degree).  "_dev" pointers are device pointers on the current
 *    CUDA device; "_host" pointers are host pointers (pinned memory gives the
 *    fastest copies, pageable memory works).  The caller owns every I/O buffer;
 *    input and output may alias (in-place transforms are allowed).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Device-side calls are asynchronous: they return once the work
 *    is enqueued; faults surface from cjt_sync or the next CUDA call.
 *  - A plan owns all its device tables and, by default, its workspace.  A plan
 *    with its own workspace may be in use on one stream at a time: a call on a
 *    different stream while the plan's previous work is still running returns
 *    CJT_EBUSY.  A plan built with shared_workspace holds only read-only tables
 *    and may run on any number of streams at once, from any number of host
 *    threads, each execution with its own workspace: every execution takes its
 *    own side stream and fork/join events from a per-device pool.  Distinct
 *    plans are independent and may run concurrently.
 *  - Return values: 0 (CJT_OK) on success, a negative CJT_E* code otherwise;
 *    cjt_strerror() names it.  No C++ exception crosses this boundary.
 *  - The library never falls back to a CPU path: every step of a transform
 *    runs in this library's CUDA kernels.
 */
#ifndef CJT_H
#define CJT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define CJT_OK 0
#define CJT_EINVAL (-1)      /* null pointer, N < 0, bad option value               */
#define CJT_EDOMAIN (-2)     /* alpha or beta outside [-1/2, 3/2] (Sec. 1.2, 2.1)     */
#define CJT_ENOMEM (-3)      /* device or host allocation failed                     */
#define CJT_ECUDA (-4)       /* a CUDA runtime call failed (see cjt_last_cuda_error) */
#define CJT_ETIMEOUT (-5)    /* a bounded device-side wait gave up                   */
#define CJT_EBUSY (-6)       /* plan still in use on another stream                  */
#define CJT_EUNSUPPORTED (-7)/* request outside what this library implements        */
#define CJT_EDIRECTION (-8)  /* plan was not built for the requested direction       */

/* Environment variables read by the library (all optional):
 *   CJT_TWIDDLE_CACHE_MB  MiB of twiddle tables kept cached after no plan uses them
 *                         (default 1024; see cjt_destroy)
 *   CJT_BATCH_ARENA_MB    MiB of one workspace arena of a grouped batch (default 4096;
 *                         see cjt_batch_create)
 *   CJT_BATCH_STREAMS     lanes of cjt_execute_batched and the default of
 *                         cjt_batch_create's nstreams (1..64, default 16)
 *   CJT_BATCH_NO_GROUP    set: cjt_batch_create runs every item as its own chain of
 *                         launches (the per-item path), with the same results
 *   CJT_PLAN_TRACE        set: cjt_plan prints the wall time of each planning step to
 *                         stderr, synchronising the stream after each
 *   CJT_GROUP_TRACE       set: a grouped batch prints one line per launch step to stderr
 *                         when it is issued (captured or profiled)                      */

/* precision of the scaled DCT-I/DST-I bulk (Sec. 2.1, Eq. "PNASY") */
#define CJT_FP64 0           /* everything in IEEE double                            */
#define CJT_MIXED 1          /* ASY transforms in float; Hahn coefficients, scalings,
                                recurrences, accumulation and the final DCT-I in double */
#define CJT_DFLOAT 2         /* ASY transforms and their inputs, and the stored recurrence
                                values (rec_store), in double-float arithmetic (pairs of
                                floats, about 48 significant bits, on the FP32 pipe); Hahn
                                coefficients, scalings, recurrences, accumulation and the
                                final DCT-I in double.  Meets the FP64 error bound
                                1e-12 ||c||_1 of this library's tests.                  */

/* asymptotic expansion of the plan (cjt_plan_opts.expansion) */
#define CJT_EXPANSION_AUTO 0           /* the ultraspherical formula when alpha = beta in
                                          (-1/2, 1/2), Hahn's formula otherwise            */
#define CJT_EXPANSION_HAHN 1           /* Hahn's formula for general (alpha, beta)
                                          (Eq. "Jacasy", Sec. 2.1)                        */
#define CJT_EXPANSION_ULTRASPHERICAL 2 /* alpha = beta = lambda - 1/2 (App. B.1): one
                                          cosine per term (requires alpha = beta)         */

/* values of cjt_plan_opts.overlap */
#define CJT_OVERLAP_AUTO 0
#define CJT_OVERLAP_ASY_FIRST 1
#define CJT_OVERLAP_EQUAL 2
#define CJT_OVERLAP_REC_FIRST 3

/* directions a plan is built for */
#define CJT_FWD 1
#define CJT_INV 2

/* Plan options.  Zero-initialised fields select the defaults noted. */
typedef struct {
    int M;            /* terms of Hahn's formula (Eq. "Jacasy"), 1..20; 0 -> 7            */
    double eps;       /* partition tolerance on each matrix entry (Sec. 2.2); 0 -> 2^-52   */
    int precision;    /* CJT_FP64 (default), CJT_MIXED or CJT_DFLOAT                       */
    int directions;   /* CJT_FWD | CJT_INV; 0 -> both                                      */
    double ratio;     /* block ratio alpha_N of Sec. 2.2 in (0, 1); 0 -> the paper's
                         min(1/log(N/n_M), 1/2)                                            */
    int seg_len;      /* degree-segment length of the recurrence work items; 0 -> 2048    */
    int use_asy;      /* 1 (default when 0): partition as in Sec. 2.2;
                         -1: recurrence only (no asymptotic blocks); other values:
                         CJT_EINVAL                                                        */
    int shared_workspace; /* 0: the plan owns its execution workspace (default);
                         1: it owns only its tables, and executions borrow a workspace
                         (cjt_forward_ws / cjt_inverse_ws, or the batched executor), so
                         that thousands of plans fit in device memory                      */
    int rec_store;    /* 0 (default): the recurrences run at each execution (Sec. 4.2).
                         1: the plan evaluates the recurrence part of the matrix once, with
                         the same stabilised forward recurrences, and keeps it in device
                         memory (8 bytes per recurrence step, rec_store_bytes); executions
                         then apply it with one fused multiply-add per entry.  With
                         alpha = beta the rows i > Ng/2 are not stored but folded
                         (parity_fold of cjt_plan_info)                                  */
    int expansion;    /* CJT_EXPANSION_AUTO (default), _HAHN or _ULTRASPHERICAL.  Both
                         formulas give the same transform (to rounding); the
                         ultraspherical one evaluates one cosine per term in the
                         diagonals u_m, v_m instead of m+1 (App. B.1).  With Hahn's
                         formula, alpha or beta = +-1/2 collapses each term to one cosine
                         (App. B.2-B.3) in either case.                                  */
    int grid;         /* Lobatto grid of the evaluation.  -1: the paper's, x_j = cos(pi j/N)
                         (forward) and cos(pi j/(2N)) (inverse); transforms of lengths 2N and
                         4N are then direct when N is 2^a, 3 2^a or 5 2^a, and Bluestein
                         transforms otherwise.  1: G, the least power of two >= N, in place of
                         N: x_j = cos(pi j/G) and cos(pi j/(2G)).  0 (default): G, the least
                         integer >= N of the forms 2^a, 3 2^a and 5 2^a (at most 4N/3; N itself
                         when N has one of them); transforms of lengths 3 2^b and 5 2^b take
                         one radix-3 or radix-5 step and power-of-two FFTs.  Every grid gives
                         the same map (to rounding): a polynomial of degree N <= G is
                         interpolated exactly by the inverse DCT-I on G+1 points, whose
                         coefficients above N vanish, and the (2G+1)-point Clenshaw--Curtis
                         rule is exact wherever the (2N+1)-point rule is.                 */
    int overlap;      /* scheduling of an execution's two concurrent chains, the
                         asymptotic blocks (pack, transforms; Eq. "PNASY") and the
                         recurrence (Sec. 4.2), which run on separate streams and join
                         before the combine.  The result does not depend on it (bit for
                         bit).  CJT_OVERLAP_ASY_FIRST: the asymptotic chain on a stream of
                         the highest priority, so the CTA scheduler serves it first and
                         the recurrence fills the SMs it leaves.  CJT_OVERLAP_EQUAL: both
                         at normal priority.  CJT_OVERLAP_REC_FIRST: the recurrence on a
                         stream of the highest priority.  CJT_OVERLAP_AUTO (0, default):
                         the library's choice for the plan's precision.                   */
    int seg_whole;    /* rows whose recurrence spans at most this many degrees run as one
                         work item of that length instead of seg_len segments, so the plan
                         computes no segment states for them (cheaper plans, longer items
                         at execution; for one-shot plans such as a server's).  0 (default):
                         every row is cut into segments of seg_len.  0 .. 2^23, else
                         CJT_EINVAL.                                                      */
} cjt_plan_opts;

/* Summary of a plan (for reports and tests). Sizes are per direction. */
typedef struct {
    int64_t N;
    double alpha, beta;
    int M, precision, directions;
    int64_t n_M;             /* Sec. 2.2, from the envelope g_M(pi/2)                  */
    double ratio;            /* alpha_N actually used                                   */
    int nblk_fwd, nblk_inv;  /* asymptotic blocks (grid G, grid 2G; G = grid_fwd)       */
    int64_t rec_steps_fwd;   /* sum_i J(i): recurrence steps of one forward transform
                                (with the parity fold: over the rows i <= N/2 only)     */
    int64_t rec_steps_inv;   /* sum_i min(J(i), N+1) on the 2G grid (likewise)          */
    int64_t fft_len_fwd, fft_len_inv;   /* transform lengths used by the ASY blocks:
                                           2 grid_fwd and 2 grid_inv                    */
    int64_t nfft_fwd, nfft_inv;         /* complex transforms per execution             */
    int64_t rec_items_fwd, rec_items_inv;
    int64_t device_bytes;    /* device memory owned by the plan                        */
    double plan_ms;          /* wall time of cjt_plan                                  */
    int64_t kernels_fwd, kernels_inv;   /* kernel launches of one execution              */
    int64_t workspace_bytes;            /* execution workspace one execution needs       */
    int64_t rec_store_bytes;            /* stored recurrence values (rec_store = 1)      */
    int shift_alpha, shift_beta;        /* 0 or 1: alpha - shift_alpha and beta - shift_beta
                                           lie in [-1/2, 1/2]                              */
    int expansion;                      /* CJT_EXPANSION_HAHN or _ULTRASPHERICAL (used)    */
    int64_t grid_fwd, grid_inv;         /* Lobatto grids used: x_j = cos(pi j / grid)     */
    int parity_fold;                    /* 1 when alpha = beta with rec_store: the stored
                                           recurrence covers the rows i <= Ng/2 and yields
                                           rows Ng - i by P_n(-x) = (-1)^n P_n(x)
                                           (DLMF 18.6.1), half the values and the work    */
    int overlap;                        /* CJT_OVERLAP_* used (AUTO resolved)              */
} cjt_plan_info;

/* Stages reported by cjt_get_profile (forward 0-4, inverse 5-9). */
#define CJT_STAGE_FWD_REC 0      /* Clenshaw--Smith / Reinsch recurrence           */
#define CJT_STAGE_FWD_PACK 1     /* C_{n,m} c_n scaling and packing                */
#define CJT_STAGE_FWD_FFT 2      /* DCT-I/DST-I transforms of the blocks           */
#define CJT_STAGE_FWD_COMBINE 3  /* diagonal scalings u_m, v_m and accumulation    */
#define CJT_STAGE_FWD_DCT 4      /* final inverse DCT-I                            */
#define CJT_STAGE_INV_FRONT 5    /* T_2N^T [c; 0] and Clenshaw--Curtis weights     */
#define CJT_STAGE_INV_PACK 6     /* (u_m + i v_m) g packing                        */
#define CJT_STAGE_INV_FFT 7      /* transposed DCT-I/DST-I transforms              */
#define CJT_STAGE_INV_REC 8      /* transposed (forward) recurrence                */
#define CJT_STAGE_INV_COMBINE 9  /* C_{n,m} scaling, accumulation, 1/A_n           */
#define CJT_NSTAGE 10

typedef struct cjt_plan_s *cjt_plan_t;

/* Fill *opts with the defaults.  Returns CJT_EINVAL if opts is NULL. */
int cjt_plan_opts_default(cjt_plan_opts *opts);

/*
 * Build a plan (Sec. 4 "Planification", steps 1a-1e): recurrence tables
 * (Sec. 1.2, Sec. 4.2 Lemma on r_n^b(+-1)), Hahn coefficients C_{n,m}
 * (Eq. "Cnmabasy"/"Cnmabrec"), diagonals u_m, v_m (Eq. "Jacasyuv"), the
 * partition n_M, alpha_N, K, j_k, i_k^1, i_k^2 (Sec. 2.2), transform twiddles,
 * and for the inverse the Clenshaw--Curtis weights (Eq. "CCweights") and
 * 1/A_n (Eq. "Anabasy").  Runs on `stream` and synchronises it once (the box
 * indices are read back to size the launches).  The plan belongs to the device that is
 * current at this call: every call that executes it (and every batch made of it) must
 * run with that device current, else it returns CJT_EINVAL and launches nothing.
 *   out    : receives the plan handle (NULL on failure)
 *   N      : degree, N >= 0 (N = 0 is the identity map); N <= 2^22
 *   alpha, beta : Jacobi parameters in [-1/2, 3/2] (else CJT_EDOMAIN).  The method itself
 *            works on [-1/2, 1/2]^2 (Sec. 2.1); a parameter in (1/2, 3/2] is reached from
 *            alpha - 1 (beta - 1) in the square by the two-term relation between Jacobi
 *            polynomials whose parameters differ by one (Sec. 1.2): the coefficients are
 *            converted in O(N) before the forward transform (a bidiagonal solve on the
 *            input) and after the inverse transform (a bidiagonal product on the output).
 *            Parameters below -1/2 would need the solve on the inverse transform's output,
 *            which sums its errors over all higher degrees, so they are not offered.
 *   opts   : NULL for defaults
 * Errors: CJT_EINVAL, CJT_EDOMAIN, CJT_ENOMEM, CJT_ECUDA, CJT_EUNSUPPORTED.
 */
int cjt_plan(cjt_plan_t *out, int64_t N, double alpha, double beta, const cjt_plan_opts *opts,
             void *stream);

/* Release a plan and all device memory it owns.  NULL is ignored.  The caller
 * must ensure no work using the plan is still running.
 * Memory the library keeps beyond its plans, per device: the twiddle tables, which plans of
 * the same transform lengths and precision share (tables no plan uses stay cached, least
 * recently used freed first, up to CJT_TWIDDLE_CACHE_MB, default 1024 MiB), and a pool of
 * plan-building temporaries that keeps up to 1 GiB of freed memory for the next plans.  A
 * plan's device_bytes (cjt_get_info) counts the shared tables it uses. */
void cjt_destroy(cjt_plan_t plan);

/* Copy the plan summary into *info. */
int cjt_get_info(cjt_plan_t plan, cjt_plan_info *info);

/*
 * Stated error bound of the plan's transform in `direction`, per unit ||c_in||_1 of the
 * input: max_k |c_k - c_k^exact| <= *bound * ||c_in||_1.
 *   CJT_FP64, CJT_DFLOAT: 1e-12, the bound this library states and tests for its FP64
 *       arithmetic (the paper bounds the inverse pessimistically, Sec. 3.3).
 *   CJT_MIXED: 1e-12 plus a bound on what the FP32 transforms of the asymptotic blocks
 *       add, derived at plan time from the componentwise error of an FP32 transform of
 *       length L, eps_F = 2^-24 (3 log2 L + 8) times the sum of its inputs' moduli, carried
 *       through the scaled items and the diagonals (Eq. "Jacasyuv"):
 *         forward: 2 eps_F max_i sum_m (|u_m| + |v_m|)(theta_i) (C_{j_k,m} + paired item),
 *         inverse: eps_F max_n (1/A_n) sum_m C_{n,m} sum_{i in box} w_i (|u_m| + |v_m|)(theta_i)
 *                  (+ paired item),
 *       with the boxes, j_k and C_{n,m} of the plan's partition (Sec. 2.2), the
 *       Clenshaw--Curtis weights w_i (Eq. "CCweights") and 1/A_n (Eq. "Anab"): the growth
 *       of 1/A_n with n is why the inverse's bound exceeds the forward's.
 * Errors: CJT_EINVAL (null, bad direction), CJT_EDIRECTION.
 */
int cjt_error_bound(cjt_plan_t plan, int direction, double *bound);

/*
 * The plan's partition (Sec. 2.2) on the grid of `direction` (x_i = cos(pi i / Ng), Ng the
 * forward grid or twice the inverse one, grid_fwd / grid_inv of cjt_plan_info): block k
 * (k = 1..nblk, outermost first) is the box of degrees [j_k, j_{k-1}) (j_0 = N+1) and rows
 * [i_k^1, i_k^2], where the asymptotic formula's remainder bound 2 C_{j_k,M} g_M(theta_i) is
 * below eps on every row; boxes[3(k-1) + 0..2] = j_k, i_k^1, i_k^2 (int64, cap blocks room).
 * With alpha = beta and stored recurrence values the boxes are the ones after the parity
 * fold (symmetric about the middle row).  *nblk receives the number of blocks.
 * Errors: CJT_EINVAL (null pointer, cap < 0, bad direction, or more than cap blocks, with
 * *nblk set), CJT_EDIRECTION.
 */
int cjt_get_partition(cjt_plan_t plan, int direction, int cap, int64_t *boxes, int *nblk);

/*
 * Forward transform (Eq. "CJT"): c_cheb_dev[k], k = 0..N, from c_jac_dev[n].
 * Both are device arrays of N+1 doubles; they may alias.
 * Errors: CJT_EINVAL (null, another device current), CJT_EDIRECTION, CJT_EBUSY, CJT_ECUDA.
 */
int cjt_forward(cjt_plan_t plan, const double *c_jac_dev, double *c_cheb_dev, void *stream);

/*
 * Inverse transform (Eq. "iCJT" through Eq. "CJTT"): c_jac_dev from c_cheb_dev.
 * Both are device arrays of N+1 doubles; they may alias.
 * Errors: CJT_EINVAL (null, another device current), CJT_EDIRECTION, CJT_EBUSY, CJT_ECUDA.
 */
int cjt_inverse(cjt_plan_t plan, const double *c_cheb_dev, double *c_jac_dev, void *stream);

/*
 * Jacobi-to-Jacobi conversion (Sec. 5: composing the forward and the inverse transform
 * converts between Jacobi bases of different parameters):
 *   c_out = P_N^{(gamma,delta)}^{-1} P_N^{(alpha,beta)} c_in,
 * the coefficients, in the basis of plan `to` (parameters gamma, delta), of the
 * polynomial of degree <= N whose coefficients in the basis of plan `from` (alpha, beta)
 * are c_in.  Runs the forward transform of `from` into c_out, then the inverse transform
 * of `to` in place on c_out, on `stream`.  c_in and c_out are device arrays of N+1
 * doubles and may alias.  Both plans must own their workspace.
 * Errors: CJT_EINVAL (null, plans of different N, shared-workspace plans),
 * CJT_EDIRECTION (`from` without CJT_FWD or `to` without CJT_INV), and those of
 * cjt_forward / cjt_inverse.
 */
int cjt_jacobi_to_jacobi(cjt_plan_t from, cjt_plan_t to, const double *c_in_dev, double *c_out_dev, void *stream);

/*
 * Forward / inverse transform with a caller-supplied workspace: workspace_dev is
 * a device buffer of at least cjt_plan_info.workspace_bytes bytes (256-byte
 * aligned), used only for the duration of the call's work on `stream`.
 * Works for every plan; required for plans built with shared_workspace = 1
 * (cjt_forward / cjt_inverse return CJT_EINVAL for those).
 */
int cjt_forward_ws(cjt_plan_t plan, const double *c_jac_dev, double *c_cheb_dev, void *workspace_dev,
                   size_t workspace_bytes, void *stream);
int cjt_inverse_ws(cjt_plan_t plan, const double *c_cheb_dev, double *c_jac_dev, void *workspace_dev,
                   size_t workspace_bytes, void *stream);

/*
 * End-to-end transform from host memory: copies in_host (N+1 doubles) to the
 * plan's device staging buffer, runs the forward (direction = CJT_FWD) or
 * inverse (CJT_INV) transform, copies the result to out_host and waits for
 * the stream.  in_host and out_host may alias.
 */
int cjt_execute_host(cjt_plan_t plan, int direction, const double *in_host, double *out_host,
                     void *stream);

/*
 * Batched execution (Sec. 4: one plan machinery applied to many inputs):
 * item t uses plans[t] in direction dir[t] (CJT_FWD or CJT_INV) on
 * in_dev + offsets[t] -> out_dev + offsets[t] (N_t + 1 doubles each, N_t the
 * degree of plans[t]).  Items may mix N, (alpha, beta), precision and
 * direction.  The items are spread, longest first, over a set of internal
 * streams that fork from and join back to `stream` through events, so the
 * call is ordered like any other work on `stream`.  Plans built with
 * shared_workspace borrow per-stream workspace arenas owned by the library,
 * grown on demand by calls that are not under stream capture (a call under
 * capture that would need a larger arena returns CJT_EBUSY).  An outgrown arena
 * is kept, not freed, until the process exits, so that a graph captured from an
 * earlier call stays valid.  A plan may appear at most once per call; in_dev
 * and out_dev must not overlap.  Every plan must belong to the current device.
 * Errors: CJT_EINVAL, CJT_EDIRECTION, CJT_EBUSY, CJT_ECUDA, CJT_ENOMEM.
 */
int cjt_execute_batched(int count, const cjt_plan_t *plans, const int8_t *dir, const int64_t *offsets,
                        const double *in_dev, double *out_dev, void *stream);

/*
 * A captured batch: cjt_batch_create captures the whole batched execution of the
 * given items and buffers into one CUDA graph and instantiates it; cjt_batch_launch
 * replays it on `stream` with a single graph launch.  Plans and buffers must outlive
 * the batch.  cjt_batch_info reports the kernel launches of one replay and the bytes
 * of the batch's private workspace arenas.  cjt_batch_launch (and _host) return
 * CJT_EINVAL unless the plans' device is current.
 *   Grouped execution (Sec. 4: one plan machinery over many coefficient sets): items
 * in FP64 or the mixed form whose transform lengths are 2^b, 3 2^b or 5 2^b (no
 * Bluestein transform) and with no parameter shift run stage by stage, one launch per
 * stage over many items, and one batched FFT per (length, precision) class.  The items
 * are taken by decreasing cost and packed into waves whose workspace fits
 * CJT_BATCH_ARENA_MB MiB (environment, default 4096); consecutive waves alternate
 * between two such arenas and two pairs of streams.  Every grouped item's result is
 * bit-identical to the same plan run alone.  The other items (double-float form,
 * shifted parameters, Bluestein lengths) run one chain of launches each over
 * `nstreams` lanes (0 -> 16).
 */
typedef struct cjt_batch_s *cjt_batch_t;
int cjt_batch_create(cjt_batch_t *out, int count, const cjt_plan_t *plans, const int8_t *dir,
                     const int64_t *offsets, const double *in_dev, double *out_dev, int nstreams);
int cjt_batch_launch(cjt_batch_t batch, void *stream);
int cjt_batch_info(cjt_batch_t batch, int64_t *kernels, int64_t *arena_bytes);
void cjt_batch_destroy(cjt_batch_t batch);

/*
 * End-to-end batched execution from host memory: copies in_host (the batch's whole input,
 * offsets as given to cjt_batch_create) to the batch's device input buffer, replays the
 * batch, copies its device output buffer to out_host and waits for `stream`.  Both host
 * arrays hold max_t (offsets[t] + N_t + 1) doubles (pinned memory gives the fastest
 * copies).  Errors: CJT_EINVAL (null), CJT_ECUDA.
 */
int cjt_batch_launch_host(cjt_batch_t batch, const double *in_host, double *out_host, void *stream);

/*
 * Batch profiling.  With cjt_batch_set_profiling(batch, 1), cjt_batch_launch issues the
 * grouped items' kernels directly, one after another on one stream (the same kernels and
 * results as a replay of its graph, without the overlap of its streams), with a CUDA event
 * pair around every launch, and cjt_batch_get_profile waits for them and returns per stage
 * kind s < n the summed milliseconds ms[s] and the launches counts[s] since the last call
 * (either pointer may be NULL).  Items that run one chain each (see cjt_batch_create) run
 * as in a replay and are not timed.
 */
#define CJT_BSTAGE_FFT_ASY 0      /* DCT-I/DST-I of the asymptotic blocks (Eq. "PNASY", "CJTT") */
#define CJT_BSTAGE_FFT_DCT 1      /* final DCT-I and the inverse front end                       */
#define CJT_BSTAGE_REC 2          /* recurrences at execution (Sec. 4.2)                         */
#define CJT_BSTAGE_REC_STORED 3   /* stored recurrence values (rec_store)                        */
#define CJT_BSTAGE_REDUCE 4       /* fixed-order sums over the transposed recurrence's items     */
#define CJT_BSTAGE_PACK 5         /* C_{n,m} c_n and (u_m + i v_m) g packing                     */
#define CJT_BSTAGE_COMBINE 6      /* accumulation of the asymptotic terms, 1/A_n                 */
#define CJT_BSTAGE_OTHER 7        /* front-end packing, Clenshaw--Curtis weights, DCT scaling    */
#define CJT_NBSTAGE 8
int cjt_batch_set_profiling(cjt_batch_t batch, int on);
int cjt_batch_get_profile(cjt_batch_t batch, double *ms, int64_t *counts, int n);

/*
 * Stage profiling.  cjt_set_profiling(plan, 1) makes every later execution of
 * the plan run its stages one after another on the launching stream (the
 * asymptotic chain no longer overlaps the recurrence) and record a CUDA event
 * pair around each stage, so that each pair times its stage alone;
 * cjt_get_profile waits for those events and returns, per stage s < n, the
 * summed milliseconds ms[s] and the number of timed launches counts[s]
 * (either pointer may be NULL), then clears the record.  Results are the same
 * bit for bit.  Profiling is off by default.
 */
int cjt_set_profiling(cjt_plan_t plan, int on);
int cjt_get_profile(cjt_plan_t plan, double *ms, int64_t *counts, int n);

/*
 * Peak arithmetic microbenchmark (diagnostic, no counterpart in the paper):
 * dependent-chain multiply-adds on every SM in FP32 (kind = 0), FP64 (kind = 1)
 * or double-float arithmetic (kind = 2: x <- x*a + b with a double-float product
 * and sum, the operations of the CJT_DFLOAT transforms).  Writes the measured rate
 * in FLOP/s to *flops (2 per multiply-add).  Other kinds: CJT_EINVAL.
 */
int cjt_microbench_fma(int kind, double *flops, void *stream);

/*
 * Transform launch configuration (for the autotuner; no counterpart in the paper).  The
 * DCT-I/DST-I sums of every stage run as batched complex FFTs of power-of-two length L;
 * per precision (CJT_FP64, CJT_MIXED: float, CJT_DFLOAT: double-float) and log2 L:
 *   ctas_per_sm      CTAs per SM the tile size (sequences per CTA) aims at (1..32, default 4);
 *   split            four-step factorisation L = L1 L2 above one pass: 0 (default) the larger
 *                    factor first (L1 = 2^ceil(log2 L / 2)), 1 the smaller first, 2 a first
 *                    factor smaller by one more power of two (L1 = 2^(floor(log2 L / 2) - 1):
 *                    the strided first pass then reads wider runs of adjacent columns; taken
 *                    only where the second pass stays within one shared-memory pass, else 0);
 *   single_max_log2  12 (default) or 13: longest transform run in one shared-memory pass.
 * The configuration holds for the process and for every later launch (a captured graph keeps
 * the configuration of its capture).  ctas_per_sm changes only the work split; split and
 * single_max_log2 change the order of the arithmetic, so results differ in rounding between
 * configurations (within the tolerances).  Errors: CJT_EINVAL.
 * cjt_fft_time runs `batch` transforms of length 2^log2L (log2L <= 22, at most 8 GB of data)
 * under the current configuration and stores the average milliseconds of `reps` runs after a
 * warm-up (CUDA events on `stream`); it allocates and frees its own buffers.
 */
int cjt_fft_set_config(int precision, int log2L, int ctas_per_sm, int split, int single_max_log2);
int cjt_fft_get_config(int precision, int log2L, int *ctas_per_sm, int *split, int *single_max_log2);
int cjt_fft_time(int precision, int log2L, int64_t batch, int reps, double *ms, void *stream);

/*
 * Allocation-free Chebyshev coefficients from values (no counterpart in the
 * paper; it is the forward transform's last step, c = T_N^{-1} y, offered for
 * callers that cannot call cudaMalloc: code running under a host framework's
 * pool allocator that owns the device memory, latency-critical paths where an
 * allocation may block or synchronise the device, and plug-ins whose host has
 * reserved nearly all device memory).
 *   values_dev : device array of N+1 doubles, y_j at x_j = cos(pi j/N)
 *   c_cheb_dev : device array of N+1 doubles receiving c_k with y_j = sum_k c_k T_k(x_j)
 * Needs no plan and allocates nothing: its working memory is a fixed device
 * array of 3 * 2 * CJT_NOALLOC_MAX_N complex doubles (6 MiB), reserved on every
 * GPU that loads the library until the process exits.  N must be 0 or a power
 * of two no larger than CJT_NOALLOC_MAX_N, else CJT_EUNSUPPORTED; CJT_EINVAL for
 * null pointers or N < 0.  The first call on a device looks up the array's
 * address on that device; make it before capturing a stream into a graph.  All
 * calls share the array: calls whose work overlaps on the GPU (other streams or
 * threads) race and must be serialised by the caller.
 */
#define CJT_NOALLOC_MAX_N 65536
int cjt_cheb_coeffs_noalloc(int64_t N, const double *values_dev, double *c_cheb_dev, void *stream);

/*
 * The plan's asymptotic expansion on the host (no GPU; for tests and reports).  The
 * expansion is the one cjt_plan picks for (alpha, beta) in [-1/2, 1/2]^2 and the
 * CJT_EXPANSION_* option `expansion`.
 *   cjt_asy_coefficient: *C = C_{n,m} (Eq. "Cnmab" for Hahn's formula, App. B.1 for the
 *       ultraspherical one), as the plan computes it (Eq. "Cnmabasy"/"Cnmabrec").
 *   cjt_asy_eval: at theta = pi i / Ng with 0 < i < Ng,
 *       *value = sum_{m<M} C_{n,m} [u_m(theta) cos(n theta) + v_m(theta) sin(n theta)]
 *       (Eq. "Jacasyuv"), the M-term approximation of P_n^{(alpha,beta)}(cos theta), and
 *       *bound = 2 C_{n,M} g_M(theta), the bound on its remainder that the partition uses
 *       (Sec. 2.2; App. B.1: 2 C^lambda_{n,M} / sin^{M+lambda} theta).
 * Errors: CJT_EINVAL (null pointer, n < 0, m outside 0..20, M outside 1..20, Ng outside
 * [2, 2^30], i outside (0, Ng), an ultraspherical request with alpha != beta),
 * CJT_EDOMAIN (alpha or beta outside [-1/2, 1/2]).
 */
int cjt_asy_coefficient(double alpha, double beta, int expansion, int64_t n, int m, double *C);

/*
 * The plan's recurrence-table entries for degree n on the host (no GPU; for tests and
 * reports), computed by the same function as the plan kernel that fills the tables.
 * out[0..CJT_REC_COEFFS-1] receives, in this order:
 *   A_n, B_n, C_n   three-term recurrence P_{n+1} = (A_n x + B_n) P_n - C_n P_{n-1}
 *                   (Sec. 1.2; n = 0: A_0 = (a+b+2)/2, B_0 = (a-b)/2, C_0 = 0);
 *   r^f_n(+1), r^f_n(-1)   forward ratios P_{n+1}(x0)/P_n(x0) of the modified forward
 *                   recurrence (Sec. 4.2);
 *   r^b_n(+1), r^b_n(-1)   backward ratios of the modified Clenshaw--Smith algorithm
 *                   (Lemma of Sec. 4.2; 0 at n = 0, where the ratio is infinite);
 *   C_n / r^f_{n-1}(+1), C_n / r^f_{n-1}(-1)   (0 at n = 0);
 *   C_n r^b_n(+1), C_n r^b_n(-1)               (0 at n = 0).
 * Errors: CJT_EINVAL (null out, n < 0 or n > 2^40), CJT_EDOMAIN (alpha or beta outside
 * [-1/2, 1/2]; plans for parameters above 1/2 use the tables of alpha - 1 or beta - 1).
 */
#define CJT_REC_COEFFS 11
int cjt_rec_coefficients(double alpha, double beta, int64_t n, double *out);
int cjt_asy_eval(double alpha, double beta, int expansion, int M, int64_t n, int64_t i, int64_t Ng, double *value,
                 double *bound);

/* Wait for `stream` and report any CUDA error raised by earlier work. */
int cjt_sync(void *stream);

/* Message for an error code (static string). */
const char *cjt_strerror(int code);

/* The last CUDA error string seen by the library on this thread ("" if none). */
const char *cjt_last_cuda_error(void);

/* Library version string. */
const char *cjt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CJT_H */
