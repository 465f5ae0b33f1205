/*
 * afmm.h -- C ABI of libafmm, a GB300 (sm_103a) implementation of the cylindrical-
 * coordinate Fast Multipole Method of M. J. Carley, "A Fast Multipole Method for
 * axisymmetric domains" (arXiv 2301.01179).
 *
 * Problem (Sec. 2, Eq. analysis:sum): given ring sources at (r_i, z_i), i = 1..Ns, with
 * Fourier coefficients S_i^(n), n = 0..N, and field points (r_j, z_j), j = 1..Nf, evaluate
 *     Phi^(n)(r_j, z_j) = sum_i S_i^(n) G^(n)(r_j, r_i, z_j - z_i),   n = 0..N,
 * with the modal Green's function (Eq. analysis:gfunc, Appendix A)
 *     G^(n)(r, r1, x) = Q_{n-1/2}(chi) / (2 pi sqrt(r r1)),  chi = (r^2 + r1^2 + x^2)/(2 r r1).
 * Only n >= 0 is computed: the source is real, so S^(-n) = conj(S^(n)) (Sec. 2).
 *
 * Conventions for every entry point:
 *  - All array arguments are DEVICE pointers (cudaMalloc'd or torch CUDA storage) to
 *    IEEE float64 data, unless a comment says otherwise.  The caller owns them.
 *  - Amplitude and result arrays are mode-major planes with real and imaginary parts in
 *    separate arrays: q_re[n * ns + i] is Re S_i^(n); phi_re[n * nf + j] is Re Phi^(n)_j.
 *    Points stay in the caller's order.
 *  - Radii must be finite and > 0 (the kernel divides by sqrt(r r1)); z must be finite.
 *  - Work is enqueued on the CUDA stream bound to the plan (or passed explicitly) and is
 *    asynchronous: the caller synchronises before reading results.  Plan creation
 *    synchronises its stream once (it reads the tree depth back to the host).
 *  - Nothing aborts or throws: every call returns an afmm_status.  A coincident source and
 *    field point (rho_- = 0, the logarithmic singularity of Appendix A) contributes 0.
 */
#ifndef AFMM_H
#define AFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AFMM_OK = 0,
    AFMM_EINVAL = 1,       /* bad size, option, NULL pointer, r <= 0 or non-finite coordinate */
    AFMM_ENOMEM = 2,       /* device allocation failed */
    AFMM_ECUDA = 3,        /* a CUDA call or kernel launch failed (see afmm_last_cuda_error) */
    AFMM_ETIMEOUT = 4,     /* a bounded device-side wait (the MMA completion barrier of the
                              tensor-core S2L, or a producer/consumer hand-over of the
                              near-field kernel) ran out during an earlier evaluation on this
                              plan; that evaluation's results are invalid.  Reported once, by
                              the next call on the plan. */
    AFMM_EUNSUPPORTED = 5  /* valid request the library does not implement (e.g. depth > 16) */
} afmm_status;

typedef enum {
    AFMM_FP64 = 0,        /* FP64-accurate results (parity 1e-10 with an FP64 reference): FP64
                             where precision demands it, FP32-pair ("double-float") arithmetic
                             where it is exact enough and faster on GB300 (near field, L2P), and
                             the S2L contraction on the bf16 tensor cores by exact 8-bit digit
                             slicing (48-bit operands, see s2l_engine) */
    AFMM_MIXED = 1,       /* FP64-class Legendre recursion and elliptic start values (FP32
                             pairs); FP32 products with compensated FP32 sums; FP32 moments and
                             locals (Sec. 2 with scaled coordinates, Eq. gfunc:scaled); S2L on
                             the tensor cores with 4-digit (32-bit) slicing */
    AFMM_FP64_NATIVE = 2  /* every floating-point operation of the path in native FP64 */
} afmm_precision;

/* Options of the FMM (Sec. 3, Algorithm 1).  Zero-initialise and set what you need;
 * afmm_options_default() fills the defaults. */
typedef struct {
    int order;          /* expansion order M (moments i+j <= M, locals k+l <= M); 0..16
                           (larger orders: AFMM_EUNSUPPORTED) */
    int leaf_size;      /* depth rule: smallest d >= 2 whose non-empty leaves hold at most
                           leaf_size sources on average; >= 1 (adaptive tree: the split
                           threshold, see tree) */
    int depth_override; /* 0: use the leaf_size rule; 2..16: use this depth (adaptive tree:
                           the maximum level, 0: 16) */
    int precision;      /* afmm_precision */
    double fwd_switch;  /* Legendre recursion: forward iff 2 N acosh(chi) <= fwd_switch.
                           AFMM_FP64_NATIVE (0: default 9 for N <= 16, 9 - 1.5 log2(N/16)
                           above, which keeps the forward sweep's error growth below
                           ~2e-12); FP32-pair kernels (AFMM_FP64, AFMM_MIXED): at most 8
                           (0: 8), and forward only while acosh(chi) <= 0.96.  The paper's
                           fixed switch is chi < 1.008 (Appendix A). */
    int miller_extra;   /* Miller start (0: 15).  AFMM_FP64_NATIVE: L = N + ceil(miller_extra /
                           acosh(chi)) + 2.  FP32-pair kernels (AFMM_FP64, AFMM_MIXED):
                           L = N + 2 + max(0, ceil(miller_extra / acosh(chi) - N / 2)), which
                           keeps the error of every mode below e^(-2 miller_extra) times the
                           pair's G^(0) */
    int s2l_engine;     /* AFMM_FP64 and AFMM_MIXED. 0: S2L (Eq. analysis:s2l) on the tcgen05
                           tensor cores when the order allows (AFMM_FP64: order <= 12,
                           AFMM_MIXED: order <= 14), else on CUDA cores; 1: always on CUDA
                           cores (FP32 pairs for AFMM_FP64, FP32 for AFMM_MIXED) */
    int tree;           /* afmm_tree.  AFMM_TREE_UNIFORM (0): the paper's uniform quadtree of
                           depth d (Sec. 2.1, Algorithm 1).  AFMM_TREE_ADAPTIVE (1): the same
                           expansions on a tree refined only where points are dense: every
                           box of levels 0..1 is split, and a box of level l >= 2 is split
                           while it holds more than leaf_size sources or more than leaf_size
                           field points and l < the maximum level (depth_override, 0: 16).
                           Each box of level >= 2 takes the S2L from the same-level boxes of
                           its interaction list (the uniform list restricted to the boxes
                           that exist); a leaf's field points take its local expansion plus
                           the direct sum over (a) the sources of the existing boxes of the
                           3 x 3 block around the leaf at its level, whole subtrees included,
                           and (b) the sources of every coarser leaf adjacent to the leaf's
                           ancestor at that leaf's level.  (a) and (b) are the U, W and X
                           lists of the standard adaptive FMM, the W and X pairs summed
                           directly; every (field point, source) pair is still covered once.
                           AFMM_FP64 and AFMM_MIXED only (AFMM_FP64_NATIVE: EUNSUPPORTED). */
    int balance;        /* adaptive tree: also split a box (below the maximum level) when a
                           same-level neighbour holds more than balance x leaf_size sources
                           or field points (0: 4; negative: off).  It bounds the direct sums
                           of every leaf by (9 balance + 8 (level - 2)) x leaf_size points of
                           the other role; without it a sparse coarse leaf touching a dense
                           box sums that box's whole subtree directly. */
} afmm_options;

typedef enum { AFMM_TREE_UNIFORM = 0, AFMM_TREE_ADAPTIVE = 1 } afmm_tree;

typedef struct afmm_plan_s *afmm_plan;

/* Plan metadata (host struct filled by afmm_plan_info). */
typedef struct {
    int depth;          /* tree depth d (adaptive tree: the deepest level that holds a leaf) */
    int n_modes;        /* N + 1 */
    int order;          /* M */
    int precision;
    double r0, z0, side;        /* domain square [r0, r0+side] x [z0, z0+side] */
    int64_t ns, nf;
    int64_t n_boxes[17];        /* boxes holding sources or field points, per level */
    int64_t near_pairs;         /* (field point, source) pairs summed directly by the FMM */
    int64_t s2l_pairs;          /* (field box, source box) S2L applications, all levels */
    int64_t expansions;         /* Green's-function expansions generated per evaluation */
    int64_t s2l_point_pairs;    /* (field point, source) pairs covered by those S2L box pairs;
                                   every pair of points is covered once, by the near field or
                                   by one level's interaction list (Sec. 2.2), so
                                   near_pairs + s2l_point_pairs = ns * nf */
    int s2l_tensor_cores;       /* 1 if the S2L runs on the tcgen05 tensor cores, else 0 */
    int tree;                   /* afmm_tree of the plan */
    int64_t n_leaves[17];       /* leaf boxes per level (uniform tree: all boxes of level d) */
    int64_t near_max_sources;   /* the most sources one leaf with field points sums directly */
} afmm_plan_info_t;

void afmm_options_default(afmm_options *opt);

/* Build a plan over sources (src_r, src_z)[ns] and field points (tgt_r, tgt_z)[nf]:
 * validates the coordinates on the device, sorts both point sets by Morton key into a
 * quadtree over the square domain (uniform: chooses the depth, Sec. 2.1 and Algorithm 1,
 * first two steps; or adaptive, see afmm_options.tree), and allocates all scratch the
 * evaluations need, so that afmm_eval, afmm_grad, afmm_direct and afmm_adjoint allocate
 * nothing.  Plan memory comes from a library-owned stream-ordered pool per device, which
 * keeps released memory reserved for the next plan: up to half the device's memory, at most
 * 128 GiB, or AFMM_POOL_KEEP_GB (environment, read when the device's pool is made).  The plan
 * copies the coordinates (the caller may free them) and is bound to `stream` (cudaStream_t,
 * NULL = legacy default stream).  n_modes = N + 1 >= 1.
 * Errors: EINVAL (ns < 1, nf < 1, n_modes < 1, bad options, NULL pointers, non-finite or
 * r <= 0 coordinates), ENOMEM, ECUDA, EUNSUPPORTED (depth > 16 required, or the adaptive
 * tree with AFMM_FP64_NATIVE). */
afmm_status afmm_plan_create(afmm_plan *out, int64_t ns, const double *src_r, const double *src_z,
                             int64_t nf, const double *tgt_r, const double *tgt_z, int n_modes,
                             const afmm_options *opt, void *stream);

/* Release the plan and its device memory (synchronises the plan's stream). NULL is ignored. */
void afmm_plan_destroy(afmm_plan p);

afmm_status afmm_plan_info(afmm_plan p, afmm_plan_info_t *info);

/* FMM evaluation of Eq. analysis:sum by Algorithm 1: leaf moments (Eq. analysis:moments),
 * upward shifts (Eq. analysis:shift), per level the local shift (Eq. analysis:l2l) and the
 * FO/BO/FI/BI source-to-local operators (Eq. analysis:s2l, Sec. 2.2) built from
 * Green's-function expansions per radial station, then local expansions plus direct
 * near-neighbour sums at the field points.  q: [n_modes][ns]; phi: [n_modes][nf]. */
afmm_status afmm_eval(afmm_plan p, const double *q_re, const double *q_im, double *phi_re,
                      double *phi_im);

/* As afmm_eval, plus the field gradient dPhi/dr and dPhi/dz at the field points (from the
 * first derivatives of G, Appendix A, in the near field and the derivative of the local
 * expansion in the far field).  phi_re/phi_im may be NULL. All outputs [n_modes][nf]. */
afmm_status afmm_grad(afmm_plan p, const double *q_re, const double *q_im, double *phi_re,
                      double *phi_im, double *dr_re, double *dr_im, double *dz_re, double *dz_im);

/* Direct O(Ns Nf) evaluation of Eq. analysis:sum over all pairs (the paper's reference
 * method, Sec. 4).  Layouts as afmm_eval. */
afmm_status afmm_direct(afmm_plan p, const double *q_re, const double *q_im, double *phi_re,
                        double *phi_im);

/* Direct evaluation with field gradient; phi_re/phi_im may be NULL. */
afmm_status afmm_direct_grad(afmm_plan p, const double *q_re, const double *q_im, double *phi_re,
                             double *phi_im, double *dr_re, double *dr_im, double *dz_re,
                             double *dz_im);

/* Adjoint of afmm_eval for a real loss L(Phi).  Input gphi = dL/dRe(Phi) + i dL/dIm(Phi)
 * ([n_modes][nf]; for L = sum |Phi - T|^2 it is 2 (Phi - T)).  Outputs:
 *   gq = dL/dRe(S) + i dL/dIm(S)            [n_modes][ns]
 *   g_src_r[i] = dL/dr_i, g_src_z[i] = dL/dz_i   [ns]
 * G is real, symmetric in r <-> r1 and even in x (Sec. 2.2), so this is the FMM on the
 * same tree with sources and field points exchanged and strengths gphi, evaluating the
 * potential A and gradient (B, C) at the sources: gq = A, dL/dr_i = sum_n Re(S conj B),
 * dL/dz_i = sum_n Re(S conj C).  Legendre recursions are recomputed, not stored. */
afmm_status afmm_adjoint(afmm_plan p, const double *q_re, const double *q_im, const double *gphi_re,
                         const double *gphi_im, double *gq_re, double *gq_im, double *g_src_r,
                         double *g_src_z);

/* Adjoint of afmm_direct (same outputs, all-pairs sums). */
afmm_status afmm_adjoint_direct(afmm_plan p, const double *q_re, const double *q_im,
                                const double *gphi_re, const double *gphi_im, double *gq_re,
                                double *gq_im, double *g_src_r, double *g_src_z);

/* Unit-level evaluators (no plan), on `stream`:
 * afmm_green: G^(n)(r[p], r1[p], x[p]) for n = 0..n_modes-1 and p < npairs, written to
 *   G[n * npairs + p] (Eq. analysis:gfunc, Legendre recursion of Eq. gfunc:recursion with
 *   start values of Eq. gfunc:Q0).  If Gr and Gx are non-NULL also dG/dr and dG/dx
 *   (Appendix A first-derivative forms).  FP64 throughout. */
afmm_status afmm_green(int64_t npairs, const double *r, const double *r1, const double *x,
                       int n_modes, double *G, double *Gr, double *Gx, void *stream);

/* afmm_green_expansion: Taylor coefficients gbar^(n)_{i,j,k}(r, r1, x) (Eq. gfunc:gnbar) for
 * i + j + k <= P, n = 0..n_modes-1, at npts points, from the x-recursion
 * (Eq. gfunc:derivatives:x), the closed first-derivative forms and the Laplace recursion
 * (Eq. gfunc:laplace).  Output dense: out[((p * n_modes + n) * (P+1) + i) * (P+1) + j) *
 * (P+1) + k], zero where i+j+k > P.  P <= 48 (AFMM_EINVAL above); AFMM_EUNSUPPORTED when the
 * per-point working set (8 (24 (P+1) + 6 n_modes (P+1) + 2 n_modes + 2 (P+1)) bytes) exceeds
 * 227 KiB of shared memory.  Requires r != r1 or x != 0 at every point.  The Legendre start
 * values and the base columns gbar_{0,0,k}, gbar_{1,0,k}, gbar_{0,1,k}, gbar_{1,1,k} are formed
 * in double-double, the rest in FP64. */
afmm_status afmm_green_expansion(int64_t npts, const double *r, const double *r1, const double *x,
                                 int n_modes, int P, double *out, void *stream);

/* afmm_fourier_analysis: azimuthal Fourier coefficients of real ring densities (Sec. 2,
 * Eq. analysis:source: s(theta) = sum_{n=-N..N} S^(n) e^{i n theta}, S^(-n) = conj(S^(n))),
 * from K equispaced samples theta_k = 2 pi k / K:
 *     S^(n) = (1/K) sum_k s(theta_k) e^{-i n theta_k},   n = 0..n_modes-1,
 * exact for band-limited densities when K >= 2 (n_modes - 1) + 1 (higher modes alias).
 * samples [K][npts] (angle-major, device); S_re, S_im [n_modes][npts] (device), the
 * amplitude layout of afmm_eval.  1 <= K <= 4096, n_modes >= 1; else AFMM_EINVAL.
 * Asynchronous on `stream`. */
afmm_status afmm_fourier_analysis(int64_t npts, int K, const double *samples, int n_modes, double *S_re,
                                  double *S_im, void *stream);

/* afmm_fourier_synthesis: the field at K equispaced angles from its modes (Sec. 2,
 * Eq. analysis:phi: phi(r, theta, z) = sum_{n=-N..N} Phi^(n) e^{i n theta}, Phi^(-n) =
 * conj(Phi^(n)) for a real field):
 *     phi(theta_k) = Re Phi^(0) + 2 sum_{n=1..n_modes-1} Re(Phi^(n) e^{i n theta_k}).
 * phi_re, phi_im [n_modes][npts] (e.g. afmm_eval's outputs, or a gradient component of
 * afmm_grad); phi [K][npts].  Same limits and errors as afmm_fourier_analysis. */
afmm_status afmm_fourier_synthesis(int64_t npts, int n_modes, const double *phi_re, const double *phi_im, int K,
                                   double *phi, void *stream);

/* afmm_direct_static: the direct sum of afmm_direct for callers that cannot allocate
 * device memory.  The paper has no counterpart; this entry point exists because some
 * callers may not call cudaMalloc: services that must keep a fixed device-memory
 * footprint after start-up, code running while another framework's caching allocator has
 * reserved nearly all device memory, and code that must avoid the device synchronisation
 * cudaMalloc/cudaFree can imply.
 *  - No plan, no allocation: the caller passes sources (src_r, src_z)[ns], field points
 *    (tgt_r, tgt_z)[nf], amplitudes q [n_modes][ns] and outputs phi [n_modes][nf] (device
 *    pointers, caller's order, same layouts as afmm_direct); the result equals
 *    afmm_direct's to rounding.
 *  - Scratch comes from one file-scope device array of AFMM_STATIC_SCRATCH_DOUBLES doubles
 *    (16 MiB) that every GPU loading this library holds until the process exits.  Requests
 *    with 2 * n_modes * ns > AFMM_STATIC_SCRATCH_DOUBLES return AFMM_EINVAL.
 *  - Every call looks the array's device address up (cudaGetSymbolAddress) in the caller's
 *    current context.  The first call in a process may load the library's device code:
 *    make it outside stream capture; later calls may be captured into a CUDA graph.
 *  - It runs the native FP64 pair kernel, not afmm_direct's FP32-pair kernel (whose extra
 *    per-point inputs do not fit the array): measured 2.8x afmm_direct's time on GB300
 *    (4096 x 4096 points, 17 modes: 12.8 ms against 4.6 ms).
 *  - Every call shares the array and leaves its contents behind; nothing is read before
 *    this call writes it.  Calls whose work overlaps on the GPU (other streams, other host
 *    threads) race on the array: serialise them.
 *  - Coordinates are not validated (radii must be finite and > 0).  Work is enqueued on
 *    `stream`. */
#define AFMM_STATIC_SCRATCH_DOUBLES 2097152
afmm_status afmm_direct_static(int64_t ns, const double *src_r, const double *src_z, int64_t nf,
                               const double *tgt_r, const double *tgt_z, int n_modes,
                               const double *q_re, const double *q_im, double *phi_re,
                               double *phi_im, void *stream);

/* Human-readable status; afmm_last_cuda_error: the last CUDA error string seen by this
 * thread's calls (static storage; "no error" if none). */
const char *afmm_status_string(afmm_status s);
const char *afmm_last_cuda_error(void);

/* Per-phase timing of the last afmm_eval / afmm_grad / afmm_adjoint on this plan, in
 * milliseconds, measured with CUDA events on the plan's stream when timing is enabled:
 * names are "perm" (strengths into sorted order), "p2m", "m2m", "gexp" (expansion
 * coefficients), "s2l", "l2l", "l2p" (local expansions at the field points), "near" (the
 * near-field sums; with AFMM_FP64_NATIVE the local expansions too, and "l2p" is empty)
 * and "total".  afmm_set_timing(p, 1) enables event recording (adds event records; the
 * evaluation waits for its last event before returning). */
afmm_status afmm_set_timing(afmm_plan p, int enable);
/* Number of CUDA kernel launches this library has made in this process (all plans and
 * unit evaluators), for accounting in benchmarks. */
long long afmm_kernel_launches(void);
afmm_status afmm_get_timing(afmm_plan p, const char *name, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* AFMM_H */
