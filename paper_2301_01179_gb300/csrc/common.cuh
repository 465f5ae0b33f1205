// common.cuh -- internal definitions shared by the libafmm translation units.
//
// Plan layout in HBM (all device arrays, FP64 unless noted):
//   sorted points   s_r, s_z [ns], t_r, t_z [nf]; s_perm, t_perm (sorted -> caller index)
//   Morton keys     s_key, t_key (uint32, level-16 interleave of (ir, iz), sorted)
//   per level l     boxes present in sources U field points, sorted by Morton key:
//                   key, src/tgt index ranges, parent, child range, 27-slot S2L table,
//                   9-slot neighbour table (leaf level), S2L work units
//   eval scratch    strengths in sorted order [n_modes][n] (pre-scaled by the Legendre
//                   recursion constants), moments and locals [box][mode][coef] per level,
//                   Green's-function expansions of one level [station][16][mode][slab]
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include "../../include/afmm.h"

#define AFMM_MAX_LEVEL 16
#define AFMM_MAX_MODES 129     // n_modes <= 129 (N <= 128)
#define AFMM_MAX_ORDER 16      // expansion order M <= 16 (S2L Taylor order 2M <= 32: two Taylor indices per lane)
#define AFMM_NEAR_WARPS 4      // warps per near-field block

namespace afmm {

// ----------------------------------------------------------------------------------------
// error handling: every CUDA call is checked; the last CUDA error string is kept per thread
// ----------------------------------------------------------------------------------------
void set_cuda_error(cudaError_t e);

#define AFMM_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            ::afmm::set_cuda_error(e_);                   \
            return e_ == cudaErrorMemoryAllocation ? AFMM_ENOMEM : AFMM_ECUDA; \
        }                                                 \
    } while (0)

void count_launch();
#define AFMM_LAUNCH_CHECK()          \
    do {                             \
        ::afmm::count_launch();      \
        AFMM_CUDA(cudaGetLastError()); \
    } while (0)

#define AFMM_TRY(expr)                                    \
    do {                                                  \
        afmm_status s_ = (expr);                          \
        if (s_ != AFMM_OK) return s_;                     \
    } while (0)

// ----------------------------------------------------------------------------------------
// Legendre recursion constants.  With G_n = c_n y_n, c_0 = c_1 = 1,
// c_n = c_{n-2} (2n-3)/(2n-1), the three-term recursion of Eq. gfunc:recursion becomes
//     y_n = gam_n chi y_{n-1} - y_{n-2}   (forward)
//     y_{n-2} = gam_n chi y_{n-1} - y_n   (backward)
// with gam_n = 4 (n-1) c_{n-1} / ((2n-3) c_{n-2}); one multiply and one FMA per step.
// The table is passed by value as a kernel argument (constant bank, warp-uniform reads).
// The backward sweep may start above N: entries run to AFMM_REC_TAB.
// ----------------------------------------------------------------------------------------
#define AFMM_REC_TAB 600
struct RecTab {
    double gam[AFMM_REC_TAB];  // gam[n], n >= 2
    double c[AFMM_MAX_MODES];  // c[n], n <= 128
};
void make_rec_tab(RecTab *t);
double default_fwd_switch(int N);

struct PairParams {
    double fwd_switch;   // forward iff 2 N acosh(chi) <= fwd_switch (and acosh(chi) <= 0.96)
    double miller_extra; // L = N + ceil(miller_extra / acosh(chi)) + 2
};

// ----------------------------------------------------------------------------------------
// quadtree
// ----------------------------------------------------------------------------------------
__host__ __device__ inline uint32_t morton_spread(uint32_t v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ inline uint32_t morton_compact(uint32_t v)
{
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}
// radial index in the odd bits, axial index in the even bits
__host__ __device__ inline uint32_t morton_key(uint32_t ir, uint32_t iz)
{
    return (morton_spread(ir) << 1) | morton_spread(iz);
}
__host__ __device__ inline uint32_t morton_ir(uint32_t k) { return morton_compact(k >> 1); }
__host__ __device__ inline uint32_t morton_iz(uint32_t k) { return morton_compact(k); }

// S2L list offsets for a field box with radial parity pr and axial parity pz: children of
// the parent's 3x3 neighbours that are not neighbours of the box (Sec. 2.2).  Slot order:
// dr from -2-pr to 3-pr, dz from -2-pz to 3-pz, skipping |dr|,|dz| <= 1.
__host__ __device__ inline void s2l_offset(int pr, int pz, int slot, int *dr, int *dz)
{
    int s = 0;
    for (int a = -2 - pr; a <= 3 - pr; ++a)
        for (int b = -2 - pz; b <= 3 - pz; ++b) {
            if (a >= -1 && a <= 1 && b >= -1 && b <= 1) continue;
            if (s == slot) {
                *dr = a;
                *dz = b;
                return;
            }
            ++s;
        }
    *dr = 0;
    *dz = 0;
}

struct Level {
    int64_t nbox = 0;
    uint32_t *key = nullptr;     // [nbox] Morton key at this level (2l bits), sorted
    int2 *srng = nullptr;        // [nbox] [begin, end) into sorted sources
    int2 *trng = nullptr;        // [nbox] [begin, end) into sorted field points
    int32_t *parent = nullptr;   // [nbox] index at level l-1 (level >= 3)
    int2 *child = nullptr;       // [nbox] child index range at level l+1 (level < d; adaptive
                                 // tree: every level, an empty range marks a leaf)
    int2 *srng_leaf = nullptr;   // adaptive tree: srng of the leaves, empty for split boxes
    int2 *trng_leaf = nullptr;   // adaptive tree: trng of the leaves, empty for split boxes
    int64_t nleaf = 0;           // leaves of this level
    int32_t *s2l = nullptr;      // [nbox][27] interaction-list box index or -1
    int32_t *nbr = nullptr;      // [nbox][9] neighbour box index or -1 (leaf level only)
    int64_t nunit = 0;           // S2L work units: up to 32 boxes of one column and parity
    int32_t *unit_box = nullptr; // [nunit][32] box indices (-1 pad)
    int32_t *unit_col = nullptr; // [nunit] column (radial index) | axial parity << 30
    int64_t nunit64 = 0;           // the same in groups of up to 64 boxes (tensor-core S2L)
    int32_t *unit64_box = nullptr; // [nunit64][64]
    int32_t *unit64_col = nullptr; // [nunit64]
    int nstation = 0;            // occupied columns
    int32_t *station_of_col = nullptr;  // [2^l] compact station index or -1
    int32_t *col_of_station = nullptr;  // [nstation]
    double *mom_re = nullptr, *mom_im = nullptr;  // [nbox][nmodes][ncoef]
    double *loc_re = nullptr, *loc_im = nullptr;  // [nbox][nmodes][ncoef]
    float *mom32_re = nullptr, *mom32_im = nullptr;  // MIXED: [nbox][nmodes][ncoef]
    float *loc32_re = nullptr, *loc32_im = nullptr;
    float2 *momd_re = nullptr, *momd_im = nullptr;   // FP64 path: FP32 pairs [nbox][nmodes][ncoef]
    float2 *locd_re = nullptr, *locd_im = nullptr;
};

// tensor-core S2L: factor tables and coefficient-index maps (host-built, passed by value)
struct TcTables {
    float2 rjl[16 * 16];      // 1 / (j! l!) as FP32 pairs, j, l <= 15
    float2 jfact[16];         // j! as FP32 pairs (a single float up to 13!)
    int8_t ci[128], cj[128];  // coefficient index -> (first, second) exponent
    // per parity pr + 2 pz: interaction-list slots in processing order, each beside its
    // axial mirror (dr, -dz); mir = 1 where a slot follows its mirror
    int8_t ord[4][27], mir[4][27];
};

// amplitude of mode n, source s: FP64 copies are planar [n][ns]; FP32 copies (MIXED) are
// per source by mode pair, [ns][npq] x (re_2m, re_2m+1, im_2m, im_2m+1), the re part at
// q = the copy, the im part at q = the copy + 2 floats
__device__ __forceinline__ double amp_at(const double *q, int n, int64_t s, int64_t ns, int npq)
{
    return q[(size_t)n * ns + s];
}
__device__ __forceinline__ float amp_at(const float *q, int n, int64_t s, int64_t ns, int npq)
{
    return q[((size_t)s * npq + (n >> 1)) * 4 + (n & 1)];
}

struct NearUnit {       // one warp of near-field work: up to 32 field points of one leaf
    int32_t box;        // leaf box index
    int32_t begin, end; // field-point range (sorted order)
    int32_t level;      // the leaf's level (d on the uniform tree)
};

// adaptive tree: a leaf's near list holds at most 9 boxes of its own level and 8 leaves of
// each coarser level >= 2 (9 + 8 x 14 for a leaf of level 16)
#define AFMM_NEAR_MAXRG 128

}  // namespace afmm

#define AFMM_EV_L2P 10  // timing event recorded between the L2P and the near-field kernel

struct afmm_plan_s {
    cudaStream_t stream = nullptr;
    int64_t ns = 0, nf = 0;
    int nmodes = 0, N = 0, M = 0, d = 0, ncoef = 0, precision = 0;
    afmm_options opt;
    afmm::PairParams pp;
    afmm::RecTab *rec = nullptr;  // host copy (passed by value to kernels)
    double r0 = 0, z0 = 0, L = 1;
    // sorted points
    double *s_r = nullptr, *s_z = nullptr, *t_r = nullptr, *t_z = nullptr;
    // sorted coordinates for the FP32-pair near field, [n][2] float4: (r0, r1, z0, z1) and
    // (r2, z2, 1/r hi, 1/r lo), r = r0 + r1 + r2 and z = z0 + z1 + z2 exactly
    float4 *s_geo = nullptr, *t_geo = nullptr;
    int32_t *s_perm = nullptr, *t_perm = nullptr;
    uint32_t *s_key = nullptr, *t_key = nullptr;
    afmm::Level lv[AFMM_MAX_LEVEL + 1];
    // near-field work units per direction (0: field points <- sources, 1: transposed)
    int64_t n_near_unit[2] = {0, 0};
    afmm::NearUnit *near_unit[2] = {nullptr, nullptr};
    // adaptive tree: per (level, box) the near list as source-role ranges, CSR over the boxes
    // of all levels (level l's boxes start at nl_base[l]; split boxes have empty lists);
    // nl_rng[0]: source ranges (field points <- sources), nl_rng[1]: field-point ranges
    int adaptive = 0;
    int64_t nl_base[AFMM_MAX_LEVEL + 2] = {0};
    int64_t *nl_off = nullptr;
    int2 *nl_rng[2] = {nullptr, nullptr};
    int nl_maxrg = 0;
    int64_t n_dir_unit[2] = {0, 0};  // direct (all pairs): units of 32 points
    afmm::NearUnit *dir_unit[2] = {nullptr, nullptr};
    // eval scratch
    double *qs_re = nullptr, *qs_im = nullptr;  // [nmodes][max(ns,nf)] strengths, sorted, * c_n
    // MIXED: the same in FP32, per point by mode pair: [n_max][n / 2]
    // (re_2m, re_2m+1, im_2m, im_2m+1)
    float4 *qs32 = nullptr;
    // FP64 path: the same as FP32 pairs, per point by mode pair, re then im:
    // [n_max][n / 2][2] (q_2m.hi, q_2m+1.hi, q_2m.lo, q_2m+1.lo)
    float4 *qsdf = nullptr;
    // FP64 path and MIXED: the L2P and near-field sums in sorted point order,
    // [6][nmodes][n_max] (potential re, im, d/dr re, im, d/dz re, im), un-permuted into the
    // caller's layout by one pass
    double *osort = nullptr;
    double df_fwd_switch = 8.0;                 // forward switch of the FP32-pair recursion
    double *gexp = nullptr;                     // expansions of one level
    double *gstart = nullptr;                   // their start values G^(n): [station][16][max(N,1)+1] double-double
    float2 *gexp_df = nullptr;                  // FP64 path: the same as FP32 pairs
    uint16_t *asl = nullptr;                    // tensor-core S2L: bf16 digit slices of the moments of one level
    afmm::TcTables *tct = nullptr;              // tensor-core S2L tables (host)
    int *err_host = nullptr, *err_dev = nullptr;  // device-side error word (mapped host memory)
    // small device-to-host reads of the tree build: a kernel writes them into mapped host
    // memory (RB_WORDS words), so they never queue behind bulk copies on the copy engines
    unsigned long long *rb_host = nullptr, *rb_dev = nullptr;
    int hw_dev = -1, hw_slot = -1;  // the plan's slot of the per-device mapped block (-1: own)
    int inject_tc_timeout = 0;                  // test hook (environment): make the S2L wait run out
    int inject_near_timeout = 0;                // test hook (environment): make a near-field hand-over run out
    int64_t gexp_cap = 0;                       // doubles
    double *m2m_tab = nullptr;                  // [4][2][(M+1)^2] shift tables (see farfield.cu)
    double *l2l_tab = nullptr;
    float2 *m2m_tab_df = nullptr, *l2l_tab_df = nullptr;  // the same as FP32 pairs
    double *acc_buf = nullptr;                  // [6][nmodes][max(ns,nf)] adjoint temporaries
    double *part_buf = nullptr;                 // direct sums split over sources: partials
    int64_t part_cap = 0;                       // doubles in part_buf
    int64_t n_max = 0;
    // statistics
    int64_t near_pairs = 0, s2l_pairs = 0, expansions = 0, s2l_point_pairs = 0;
    int64_t near_max_src = 0;  // the most sources one leaf sums directly
    // timing (events on the plan's stream; read back after the evaluation's last event)
    int timing = 0;
    cudaEvent_t ev[80];                         // phase timing events (AFMM_EV_L2P: after the L2P)
    double t_ms[9] = {0};
    // device allocations to free (from the library's stream-ordered pool when pool != null)
    cudaMemPool_t pool = nullptr;
    void *allocs[1024];
    int nalloc = 0;
};

namespace afmm {
afmm_status dalloc(afmm_plan p, void **ptr, size_t bytes);
template <typename T>
inline afmm_status dalloc_t(afmm_plan p, T **ptr, size_t count)
{
    return dalloc(p, (void **)ptr, count * sizeof(T) + 16);
}

// tree.cu
afmm_status build_tree(afmm_plan p, const double *src_r, const double *src_z, const double *tgt_r,
                       const double *tgt_z);
// nearfield.cu
afmm_status launch_near(afmm_plan p, int dir, int with_local, int grad, double *phi_re, double *phi_im,
                        double *dr_re, double *dr_im, double *dz_re, double *dz_im, int direct);
afmm_status launch_green(int64_t npairs, const double *r, const double *r1, const double *x, int n_modes,
                         double *G, double *Gr, double *Gx, cudaStream_t st);
afmm_status launch_permute(afmm_plan p, int dir, const double *q_re, const double *q_im);
constexpr int RB_WORDS = 24;
// bytes (a multiple of 8, at most 8 RB_WORDS) from device memory to host memory through the
// plan's mapped words; synchronises the plan's stream
afmm_status readback(afmm_plan p, void *host, const void *dev, size_t bytes);
// farfield.cu
afmm_status far_field(afmm_plan p, int dir);
afmm_status launch_green_expansion(int64_t npts, const double *r, const double *r1, const double *x,
                                   int n_modes, int P, double *out, cudaStream_t st);
afmm_status make_shift_tables(afmm_plan p);
// s2l_tc.cu
bool s2l_tc_enabled(afmm_plan p);
int64_t s2l_tc_slice_elems(afmm_plan p, int64_t nbox);
afmm_status make_tc_tables(afmm_plan p);
afmm_status launch_s2l_tc(afmm_plan p, int l, const double *mre, const double *mim, double *lre, double *lim);
afmm_status launch_s2l_tc(afmm_plan p, int l, const float *mre, const float *mim, float *lre, float *lim);
afmm_status launch_s2l_tc(afmm_plan p, int l, const float2 *mre, const float2 *mim, float2 *lre, float2 *lim);
}  // namespace afmm
