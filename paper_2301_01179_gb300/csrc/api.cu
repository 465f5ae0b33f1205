// api.cu -- the C ABI of libafmm (include/afmm.h): plan life cycle and the orchestration
// of Algorithm 1 (FMM), the direct sum and the adjoint on the plan's stream.
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <new>
#include "common.cuh"

namespace afmm {

static thread_local char g_cuda_err[256] = "no error";
static unsigned long long g_launches = 0;

void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }

void set_cuda_error(cudaError_t e)
{
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

// Plan memory comes from a library-owned, stream-ordered pool per device: allocation and
// release are asynchronous on the plan's stream, and up to 32 GiB of released plan memory
// stays reserved for the next plan (plain cudaMalloc/cudaFree cost milliseconds and
// synchronise the device).  Falls back to cudaMalloc when no pool can be made.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static int g_pool_state[64];  // 0: not tried, 1: ready, -1: unavailable

static cudaMemPool_t plan_pool(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (g_pool_state[dev] == 0) {
        cudaMemPoolProps pr;
        memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t pool;
        if (cudaMemPoolCreate(&pool, &pr) != cudaSuccess) {
            cudaGetLastError();
            g_pool_state[dev] = -1;
            return nullptr;
        }
        // released plan memory kept reserved for the next plan (a plan built per step, as in
        // a training loop, then reuses it instead of mapping fresh memory): half the device's
        // memory, at most 128 GiB, or AFMM_POOL_KEEP_GB
        size_t fr = 0, total = 0;
        if (cudaMemGetInfo(&fr, &total) != cudaSuccess) {
            cudaGetLastError();
            total = 64ull << 30;
        }
        uint64_t keep = total / 2 < (128ull << 30) ? total / 2 : (128ull << 30);
        if (const char *e = getenv("AFMM_POOL_KEEP_GB")) {
            const double gb = atof(e);
            if (gb >= 0.0) keep = (uint64_t)(gb * (double)(1ull << 30));
        }
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
        g_pool_state[dev] = 1;
    }
    return g_pool_state[dev] == 1 ? g_pool[dev] : nullptr;
}

// Mapped pinned host words of the plans (error word, small readbacks): one block per device,
// made once, with a 256-byte slot per live plan.  Page-locked allocations and frees
// synchronise with the work of other streams, so a plan that made its own would wait for,
// e.g., the download of an earlier result.  A plan that finds no free slot makes its own.
constexpr int HW_SLOTS = 512, HW_SLOT_BYTES = 256;
static char *g_hw_host[64], *g_hw_dev[64];
static unsigned char g_hw_used[64][HW_SLOTS];
static int g_hw_state[64];

static afmm_status hostwords_take(afmm_plan p)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        dev = -1;
    }
    char *h = nullptr, *d = nullptr;
    if (dev >= 0) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (g_hw_state[dev] == 0) {
            char *bh = nullptr, *bd = nullptr;
            cudaError_t e = cudaHostAlloc((void **)&bh, (size_t)HW_SLOTS * HW_SLOT_BYTES, cudaHostAllocMapped);
            if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&bd, bh, 0);
            if (e == cudaSuccess) {
                g_hw_host[dev] = bh;
                g_hw_dev[dev] = bd;
                g_hw_state[dev] = 1;
            } else {
                cudaGetLastError();
                g_hw_state[dev] = -1;
            }
        }
        if (g_hw_state[dev] == 1)
            for (int i = 0; i < HW_SLOTS; ++i)
                if (!g_hw_used[dev][i]) {
                    g_hw_used[dev][i] = 1;
                    p->hw_dev = dev;
                    p->hw_slot = i;
                    h = g_hw_host[dev] + (size_t)i * HW_SLOT_BYTES;
                    d = g_hw_dev[dev] + (size_t)i * HW_SLOT_BYTES;
                    break;
                }
    }
    if (!h) {
        cudaError_t e = cudaHostAlloc((void **)&h, HW_SLOT_BYTES, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&d, h, 0);
        if (e != cudaSuccess) {
            set_cuda_error(e);
            cudaGetLastError();
            return AFMM_ECUDA;
        }
    }
    memset(h, 0, HW_SLOT_BYTES);
    p->err_host = (int *)h;
    p->err_dev = (int *)d;
    p->rb_host = (unsigned long long *)(h + 64);
    p->rb_dev = (unsigned long long *)(d + 64);
    return AFMM_OK;
}

static void hostwords_give(afmm_plan p)
{
    if (!p->err_host) return;
    if (p->hw_slot >= 0) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        g_hw_used[p->hw_dev][p->hw_slot] = 0;
    } else {
        cudaFreeHost(p->err_host);
    }
    p->err_host = p->err_dev = nullptr;
}

afmm_status dalloc(afmm_plan p, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (p->nalloc >= (int)(sizeof(p->allocs) / sizeof(p->allocs[0]))) return AFMM_ENOMEM;
    void *q = nullptr;
    cudaError_t e = p->pool ? cudaMallocFromPoolAsync(&q, bytes, p->pool, p->stream) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        cudaGetLastError();
        return AFMM_ENOMEM;
    }
    p->allocs[p->nalloc++] = q;
    *ptr = q;
    return AFMM_OK;
}

void make_rec_tab(RecTab *t)
{
    static double c[AFMM_REC_TAB + 2];
    c[0] = 1.0;
    c[1] = 1.0;
    for (int n = 2; n < AFMM_REC_TAB + 2; ++n) c[n] = c[n - 2] * (2.0 * n - 3.0) / (2.0 * n - 1.0);
    for (int n = 0; n < AFMM_REC_TAB; ++n)
        t->gam[n] = n >= 2 ? 4.0 * (n - 1) * c[n - 1] / ((2.0 * n - 3.0) * c[n - 2]) : 0.0;
    for (int n = 0; n < AFMM_MAX_MODES; ++n) t->c[n] = c[n];
}

// Default forward/backward switch of the Legendre recursion on 2 N acosh(chi).  A rounding
// of size eps anywhere in the forward sweep grows to about eps N exp(2 N acosh chi) / s at
// mode N; 9 for N <= 16, then 1.5 less per doubling of N keeps that below 2e-12.
double default_fwd_switch(int N)
{
    if (N <= 16) return 9.0;
    return 9.0 - 1.5 * log2((double)N / 16.0);
}

static void tmark(afmm_plan p, int idx)
{
    if (p->timing && idx < 80) cudaEventRecord(p->ev[idx], p->stream);
}

// elapsed time between two recorded events; an event a path did not record reads as 0 and
// its error is cleared so that it cannot surface at a later launch check
static float tdiff(afmm_plan p, int a, int b)
{
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->ev[a], p->ev[b]) != cudaSuccess) {
        (void)cudaGetLastError();
        ms = 0.0f;
    }
    return ms;
}

}  // namespace afmm

using namespace afmm;

extern "C" {

void afmm_options_default(afmm_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->order = 8;
    opt->leaf_size = 32;
    opt->depth_override = 0;
    opt->precision = AFMM_FP64;
    opt->fwd_switch = 0.0;
    opt->miller_extra = 0;
    opt->s2l_engine = 0;
}

const char *afmm_status_string(afmm_status s)
{
    switch (s) {
    case AFMM_OK: return "ok";
    case AFMM_EINVAL: return "invalid argument";
    case AFMM_ENOMEM: return "out of device memory";
    case AFMM_ECUDA: return "CUDA error";
    case AFMM_ETIMEOUT: return "device wait timed out";
    case AFMM_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char *afmm_last_cuda_error(void) { return g_cuda_err; }

void afmm_plan_destroy(afmm_plan p)
{
    if (!p) return;
    if (p->pool) {
        for (int i = 0; i < p->nalloc; ++i) cudaFreeAsync(p->allocs[i], p->stream);
        cudaStreamSynchronize(p->stream);
    } else {
        cudaStreamSynchronize(p->stream);
        for (int i = 0; i < p->nalloc; ++i) cudaFree(p->allocs[i]);
    }
    hostwords_give(p);
    delete p->tct;
    if (p->timing)
        for (int i = 0; i < 80; ++i) cudaEventDestroy(p->ev[i]);
    delete p->rec;
    delete p;
}

afmm_status afmm_plan_create(afmm_plan *out, int64_t ns, const double *src_r, const double *src_z, int64_t nf,
                             const double *tgt_r, const double *tgt_z, int n_modes, const afmm_options *opt_in,
                             void *stream)
{
    if (!out) return AFMM_EINVAL;
    *out = nullptr;
    afmm_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        afmm_options_default(&opt);
    if (ns < 1 || nf < 1 || ns > 0x3fffffff || nf > 0x3fffffff) return AFMM_EINVAL;
    if (n_modes < 1 || n_modes > AFMM_MAX_MODES) return AFMM_EINVAL;
    if (!src_r || !src_z || !tgt_r || !tgt_z) return AFMM_EINVAL;
    if (opt.order < 0 || opt.leaf_size < 1 || opt.depth_override < 0 || opt.depth_override == 1 ||
        opt.depth_override > AFMM_MAX_LEVEL || opt.fwd_switch < 0.0 || opt.miller_extra < 0 ||
        (opt.s2l_engine != 0 && opt.s2l_engine != 1) ||
        (opt.tree != AFMM_TREE_UNIFORM && opt.tree != AFMM_TREE_ADAPTIVE))
        return AFMM_EINVAL;
    if (opt.precision != AFMM_FP64 && opt.precision != AFMM_MIXED && opt.precision != AFMM_FP64_NATIVE)
        return AFMM_EINVAL;
    if (opt.order > AFMM_MAX_ORDER) return AFMM_EUNSUPPORTED;
    if (opt.tree == AFMM_TREE_ADAPTIVE && opt.precision == AFMM_FP64_NATIVE) return AFMM_EUNSUPPORTED;

    afmm_plan p = new (std::nothrow) afmm_plan_s();
    if (!p) return AFMM_ENOMEM;
    p->rec = new (std::nothrow) RecTab();
    if (!p->rec) {
        delete p;
        return AFMM_ENOMEM;
    }
    make_rec_tab(p->rec);
    p->stream = (cudaStream_t)stream;
    {
        int dev = 0;
        p->pool = cudaGetDevice(&dev) == cudaSuccess ? plan_pool(dev) : nullptr;
        cudaGetLastError();
    }
    p->ns = ns;
    p->nf = nf;
    p->nmodes = n_modes;
    p->N = n_modes - 1;
    p->M = opt.order;
    p->ncoef = (opt.order + 1) * (opt.order + 2) / 2;
    p->precision = opt.precision;
    p->opt = opt;
    // failure-detection test hook: AFMM_INJECT_TC_TIMEOUT=1 makes the tensor-core S2L skip the
    // MMAs and the completion of its first slot, so that its bounded wait runs out
    {
        const char *e = getenv("AFMM_INJECT_TC_TIMEOUT");
        p->inject_tc_timeout = (e && e[0] == '1') ? 1 : 0;
        // AFMM_INJECT_NEAR_TIMEOUT=1: the near-field producers never hand over slot 0, so
        // the consumers' bounded wait on it runs out
        const char *f = getenv("AFMM_INJECT_NEAR_TIMEOUT");
        p->inject_near_timeout = (f && f[0] == '1') ? 1 : 0;
    }
    p->pp.fwd_switch = opt.fwd_switch > 0.0 ? opt.fwd_switch : default_fwd_switch(p->N);
    p->pp.miller_extra = opt.miller_extra > 0 ? (double)opt.miller_extra : 15.0;
    // FP32-pair recursion (AFMM_FP64, AFMM_MIXED): rounding ~2^-47 instead of 2^-53.  The
    // forward sweep's rounding grows like e^{n a} against the decaying Q_{n-1/2} ~ e^{-n a}
    // (a = acosh chi), so its error measured against the pair's G^(0), the scale of the
    // per-mode error max|Phi - Phi_ref| / max|Phi_ref|, is ~2^-47 N e^{s/2} / s <= 2e-12
    // for s = 2 N a <= 8 (N <= 64)
    p->df_fwd_switch = opt.fwd_switch > 0.0 ? fmin(opt.fwd_switch, 8.0) : 8.0;

    afmm_status s = hostwords_take(p);
    if (s == AFMM_OK) s = build_tree(p, src_r, src_z, tgt_r, tgt_z);
    if (s == AFMM_OK) s = make_shift_tables(p);
    // evaluation scratch: nothing is allocated by the evaluation calls
    const int nm = p->nmodes, nc = p->ncoef;
    const int64_t nmax = p->n_max;
    const bool mix = p->precision == AFMM_MIXED;
    if (s == AFMM_OK && !mix) s = dalloc_t(p, &p->qs_re, (size_t)nm * nmax);
    if (s == AFMM_OK && !mix) s = dalloc_t(p, &p->qs_im, (size_t)nm * nmax);
    const size_t npq = (size_t)(nm + 1) / 2;  // mode pairs of the interleaved amplitude copies
    if (s == AFMM_OK && mix) s = dalloc_t(p, &p->qs32, npq * nmax);
    if (s == AFMM_OK) s = dalloc_t(p, &p->acc_buf, (size_t)6 * nm * p->ns);
    int64_t gcap = 0, nexp = 0;
    for (int l = 2; s == AFMM_OK && l <= p->d; ++l) {
        Level &v = p->lv[l];
        size_t per = (size_t)v.nbox * nm * nc;
        if (mix) {
            s = dalloc_t(p, &v.mom32_re, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.mom32_im, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.loc32_re, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.loc32_im, per);
        } else if (p->precision == AFMM_FP64) {  // FP32 pairs
            s = dalloc_t(p, &v.momd_re, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.momd_im, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.locd_re, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.locd_im, per);
        } else {
            s = dalloc_t(p, &v.mom_re, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.mom_im, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.loc_re, per);
            if (s == AFMM_OK) s = dalloc_t(p, &v.loc_im, per);
        }
        int64_t g = (int64_t)v.nstation * 16 * nm * (p->M + 1) * (p->M + 1) * (2 * p->M + 1);
        if (g > gcap) gcap = g;
        nexp += (int64_t)v.nstation * 12;
    }
    p->expansions = nexp;
    // FP64 expansions (the FP64 path and the tensor-core S2L use FP32-pair expansions instead)
    const bool dfx = p->precision == AFMM_FP64 || s2l_tc_enabled(p);
    if (s == AFMM_OK && gcap > 0 && !dfx) s = dalloc_t(p, &p->gexp, gcap);
    p->gexp_cap = gcap;
    if (s == AFMM_OK) {  // start values of one level's expansions (double-double)
        int64_t smax = 1;
        for (int l = 2; l <= p->d; ++l) smax = p->lv[l].nstation > smax ? p->lv[l].nstation : smax;
        s = dalloc_t(p, &p->gstart, (size_t)smax * 16 * ((p->N < 1 ? 1 : p->N) + 1) * 2);
    }
    if (s == AFMM_OK && p->precision == AFMM_FP64) s = dalloc_t(p, &p->qsdf, 2 * npq * nmax);
    if (s == AFMM_OK && p->precision != AFMM_FP64_NATIVE) s = dalloc_t(p, &p->osort, (size_t)6 * nm * nmax);
    if (s == AFMM_OK && dfx) {
        int64_t mmax = 0;
        for (int l = 2; l <= p->d; ++l) mmax = p->lv[l].nbox > mmax ? p->lv[l].nbox : mmax;
        if (gcap > 0) s = dalloc_t(p, &p->gexp_df, gcap);
        if (s2l_tc_enabled(p)) {
            if (s == AFMM_OK) s = dalloc_t(p, &p->asl, (size_t)s2l_tc_slice_elems(p, mmax));
            if (s == AFMM_OK) s = make_tc_tables(p);
        }
    }
    // direct sums over few field points are split over sources: room for the partials
    // of up to 64 splits of the smaller point set, at most 1 GB
    if (s == AFMM_OK) {
        int64_t nmin = p->ns < p->nf ? p->ns : p->nf;
        double want = 64.0 * 6.0 * nm * (double)nmin;
        if (want > 1.25e8) want = 1.25e8;
        p->part_cap = (int64_t)want;
        s = dalloc_t(p, &p->part_buf, (size_t)p->part_cap);
    }
    if (s == AFMM_OK) {
        cudaError_t e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) {
            set_cuda_error(e);
            s = AFMM_ECUDA;
        }
    }
    if (s != AFMM_OK) {
        afmm_plan_destroy(p);
        return s;
    }
    *out = p;
    return AFMM_OK;
}

afmm_status afmm_plan_info(afmm_plan p, afmm_plan_info_t *info)
{
    if (!p || !info) return AFMM_EINVAL;
    memset(info, 0, sizeof(*info));
    info->depth = p->d;
    info->n_modes = p->nmodes;
    info->order = p->M;
    info->precision = p->precision;
    info->r0 = p->r0;
    info->z0 = p->z0;
    info->side = p->L;
    info->ns = p->ns;
    info->nf = p->nf;
    for (int l = 0; l <= AFMM_MAX_LEVEL; ++l) info->n_boxes[l] = p->lv[l].nbox;
    info->near_pairs = p->near_pairs;
    info->s2l_pairs = p->s2l_pairs;
    info->expansions = p->expansions;
    info->s2l_point_pairs = p->s2l_point_pairs;
    info->s2l_tensor_cores = s2l_tc_enabled(p) ? 1 : 0;
    info->tree = p->adaptive ? AFMM_TREE_ADAPTIVE : AFMM_TREE_UNIFORM;
    info->near_max_sources = p->near_max_src;
    for (int l = 2; l <= p->d; ++l) info->n_leaves[l] = p->adaptive ? p->lv[l].nleaf : (l == p->d ? p->lv[l].nbox : 0);
    return AFMM_OK;
}

long long afmm_kernel_launches(void) { return (long long)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

afmm_status afmm_set_timing(afmm_plan p, int enable)
{
    if (!p) return AFMM_EINVAL;
    if (enable && !p->timing) {
        for (int i = 0; i < 80; ++i) AFMM_CUDA(cudaEventCreate(&p->ev[i]));
        p->timing = 1;
    }
    return AFMM_OK;
}

afmm_status afmm_get_timing(afmm_plan p, const char *name, double *ms)
{
    if (!p || !name || !ms) return AFMM_EINVAL;
    static const char *names[] = {"perm", "p2m", "m2m", "gexp", "s2l", "l2l", "near", "total", "l2p"};
    for (int i = 0; i < 9; ++i)
        if (!strcmp(name, names[i])) {
            *ms = p->t_ms[i];
            return AFMM_OK;
        }
    return AFMM_EINVAL;
}

// a bounded device-side wait of an earlier evaluation ran out: report it once
static afmm_status take_device_error(afmm_plan p)
{
    if (p->err_host && *(volatile int *)p->err_host) {
        *(volatile int *)p->err_host = 0;
        return AFMM_ETIMEOUT;
    }
    return AFMM_OK;
}

static afmm_status run_fmm(afmm_plan p, int dir, const double *q_re, const double *q_im, int grad, double *o_re,
                           double *o_im, double *dr_re, double *dr_im, double *dz_re, double *dz_im)
{
    AFMM_TRY(take_device_error(p));
    tmark(p, 0);
    AFMM_TRY(launch_permute(p, dir, q_re, q_im));
    tmark(p, 1);
    AFMM_TRY(far_field(p, dir));
    tmark(p, 8);
    AFMM_TRY(launch_near(p, dir, 1, grad, o_re, o_im, dr_re, dr_im, dz_re, dz_im, 0));
    tmark(p, 9);
    if (p->timing) {
        AFMM_CUDA(cudaEventSynchronize(p->ev[9]));
        p->t_ms[0] = tdiff(p, 0, 1);
        p->t_ms[1] = tdiff(p, 1, 2);
        p->t_ms[2] = tdiff(p, 2, 3);
        // near: the near-field kernel after the L2P (event AFMM_EV_L2P between them)
        p->t_ms[8] = tdiff(p, 8, AFMM_EV_L2P);
        p->t_ms[6] = tdiff(p, AFMM_EV_L2P, 9);
        p->t_ms[7] = tdiff(p, 0, 9);
        double g = 0, s2 = 0, l2 = 0;
        for (int l = 2; l <= p->d; ++l) {  // per level: L2L, expansions, S2L (far_field)
            int e = 16 + 4 * (l - 2);
            l2 += tdiff(p, e, e + 1);
            g += tdiff(p, e + 1, e + 2);
            s2 += tdiff(p, e + 2, e + 3);
        }
        p->t_ms[3] = g;
        p->t_ms[4] = s2;
        p->t_ms[5] = l2;
        AFMM_TRY(take_device_error(p));
    }
    return AFMM_OK;
}

afmm_status afmm_eval(afmm_plan p, const double *q_re, const double *q_im, double *phi_re, double *phi_im)
{
    if (!p || !q_re || !q_im || !phi_re || !phi_im) return AFMM_EINVAL;
    return run_fmm(p, 0, q_re, q_im, 0, phi_re, phi_im, nullptr, nullptr, nullptr, nullptr);
}

afmm_status afmm_grad(afmm_plan p, const double *q_re, const double *q_im, double *phi_re, double *phi_im,
                      double *dr_re, double *dr_im, double *dz_re, double *dz_im)
{
    if (!p || !q_re || !q_im || !dr_re || !dr_im || !dz_re || !dz_im) return AFMM_EINVAL;
    return run_fmm(p, 0, q_re, q_im, 1, phi_re, phi_im, dr_re, dr_im, dz_re, dz_im);
}

afmm_status afmm_direct(afmm_plan p, const double *q_re, const double *q_im, double *phi_re, double *phi_im)
{
    if (!p || !q_re || !q_im || !phi_re || !phi_im) return AFMM_EINVAL;
    AFMM_TRY(launch_permute(p, 0, q_re, q_im));
    return launch_near(p, 0, 0, 0, phi_re, phi_im, nullptr, nullptr, nullptr, nullptr, 1);
}

afmm_status afmm_direct_grad(afmm_plan p, const double *q_re, const double *q_im, double *phi_re, double *phi_im,
                             double *dr_re, double *dr_im, double *dz_re, double *dz_im)
{
    if (!p || !q_re || !q_im || !dr_re || !dr_im || !dz_re || !dz_im) return AFMM_EINVAL;
    AFMM_TRY(launch_permute(p, 0, q_re, q_im));
    return launch_near(p, 0, 0, 1, phi_re, phi_im, dr_re, dr_im, dz_re, dz_im, 1);
}

// dL/dr_i = sum_n Re(S conj B), dL/dz_i = sum_n Re(S conj C)
__global__ void k_adjoint_combine(const double *__restrict__ q_re, const double *__restrict__ q_im,
                                  const double *__restrict__ acc, int nm, int64_t ns, double *__restrict__ g_r,
                                  double *__restrict__ g_z)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const size_t P = (size_t)nm * ns;
    double ar = 0.0, az = 0.0;
    for (int n = 0; n < nm; ++n) {
        size_t o = (size_t)n * ns + i;
        ar = fma(q_re[o], acc[2 * P + o], ar);
        ar = fma(q_im[o], acc[3 * P + o], ar);
        az = fma(q_re[o], acc[4 * P + o], az);
        az = fma(q_im[o], acc[5 * P + o], az);
    }
    g_r[i] = ar;
    g_z[i] = az;
}

static afmm_status run_adjoint(afmm_plan p, int direct, const double *q_re, const double *q_im,
                               const double *gphi_re, const double *gphi_im, double *gq_re, double *gq_im,
                               double *g_r, double *g_z)
{
    const size_t P = (size_t)p->nmodes * p->ns;
    double *A = p->acc_buf;
    // transposed problem: "sources" are the field points with strengths gphi, evaluated at
    // the sources with gradient
    if (direct) {
        AFMM_TRY(launch_permute(p, 1, gphi_re, gphi_im));
        AFMM_TRY(launch_near(p, 1, 0, 1, gq_re, gq_im, A + 2 * P, A + 3 * P, A + 4 * P, A + 5 * P, 1));
    } else {
        AFMM_TRY(run_fmm(p, 1, gphi_re, gphi_im, 1, gq_re, gq_im, A + 2 * P, A + 3 * P, A + 4 * P, A + 5 * P));
    }
    unsigned nb = (unsigned)((p->ns + 255) / 256);
    k_adjoint_combine<<<nb, 256, 0, p->stream>>>(q_re, q_im, A, p->nmodes, p->ns, g_r, g_z);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

afmm_status afmm_adjoint(afmm_plan p, const double *q_re, const double *q_im, const double *gphi_re,
                         const double *gphi_im, double *gq_re, double *gq_im, double *g_src_r, double *g_src_z)
{
    if (!p || !q_re || !q_im || !gphi_re || !gphi_im || !gq_re || !gq_im || !g_src_r || !g_src_z) return AFMM_EINVAL;
    return run_adjoint(p, 0, q_re, q_im, gphi_re, gphi_im, gq_re, gq_im, g_src_r, g_src_z);
}

afmm_status afmm_adjoint_direct(afmm_plan p, const double *q_re, const double *q_im, const double *gphi_re,
                                const double *gphi_im, double *gq_re, double *gq_im, double *g_src_r,
                                double *g_src_z)
{
    if (!p || !q_re || !q_im || !gphi_re || !gphi_im || !gq_re || !gq_im || !g_src_r || !g_src_z) return AFMM_EINVAL;
    return run_adjoint(p, 1, q_re, q_im, gphi_re, gphi_im, gq_re, gq_im, g_src_r, g_src_z);
}

afmm_status afmm_green(int64_t npairs, const double *r, const double *r1, const double *x, int n_modes, double *G,
                       double *Gr, double *Gx, void *stream)
{
    if (npairs < 0 || !r || !r1 || !x || !G || n_modes < 1 || n_modes > AFMM_MAX_MODES) return AFMM_EINVAL;
    if ((Gr == nullptr) != (Gx == nullptr)) return AFMM_EINVAL;
    if (npairs == 0) return AFMM_OK;
    return launch_green(npairs, r, r1, x, n_modes, G, Gr, Gx, (cudaStream_t)stream);
}

afmm_status afmm_green_expansion(int64_t npts, const double *r, const double *r1, const double *x, int n_modes, int P,
                                 double *out, void *stream)
{
    if (npts < 0 || !r || !r1 || !x || !out || n_modes < 1 || n_modes > AFMM_MAX_MODES || P < 0 || P > 48)
        return AFMM_EINVAL;
    if (npts == 0) return AFMM_OK;
    return launch_green_expansion(npts, r, r1, x, n_modes, P, out, (cudaStream_t)stream);
}

}  // extern "C"
