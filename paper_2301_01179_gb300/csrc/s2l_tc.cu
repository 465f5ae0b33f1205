// s2l_tc.cu -- the source-to-local operator (Eq. analysis:s2l, the S2L step of Algorithm 1)
// of the FP64 path on the fifth-generation tensor cores (tcgen05.mma, bf16 in, FP32 out).
//
// Per interaction-list slot, a unit of up to 64 boxes of one column and axial parity needs
//     F_kl += sum_ij  A_ij * B_kl,ij,     A_ij = j! S_ij = sum q U^i W^j,
//                                         B_kl,ij = E_{k,i,j+l} / (j! l!),
// with E the box-scaled, oriented Taylor coefficients (FO/BO/FI/BI of Sec. 2.2).  Moving
// the factorials onto B balances both operands: A decays like 2^-(i+j), and each column of
// B varies by a bounded binomial factor instead of (j+l)!.  The contraction is a GEMM:
// 128 rows (box x {re, im}) x K = ij x N = kl, padded to KP = 16 ceil(ncoef / 16) <= 96.
//
// FP64-class accuracy from bf16 tensor cores by exact digit slicing (the Ozaki scheme):
// every row of A and every column of B is written as six signed 8-bit digits on a common
// power-of-two grid of its own, a = sum_s a_s, a_s a multiple of 2^(e - 8 - 8s), with
// |a_s| <= 128 grid units (256 for s = 3, where the low FP32 word joins).  A digit is exact
// in bf16 and a digit product exact in FP32.  Level L of the product expansion, the sum of
// a_s b_t over s + t = L, is a sum of at most 4 KP products on one grid of at most 2^15
// units each: below 2^24 units for KP <= 96, so its FP32 accumulation is EXACT.
//     L0 .. L3  one accumulator per level, exact, drained after every slot into FP32-pair
//               (double-float) registers (L3, of weight 2^-24, joins the low word)
//     L4        levels 4 and 5 (weight <= 2^-32), FP32 over all slots
// An FP32 accumulation of level 2 alone would already cost ~2^-40 per product, amplified
// by the thousands of products per output; the exact levels keep the contraction at the
// FP32-pair level.  Dropped products (s + t >= 6) are below 2^-48 of the row and column
// maxima.
//
// Operands in shared memory use the no-swizzle K-major layout of 8-row x 16-byte core
// matrices; the five accumulators live in tensor memory (TMEM) columns [lv KP, (lv+1) KP).  One thread issues the MMAs; completion is tracked with mbarriers whose waits
// are bounded: a wait that runs out sets the plan's error word and the block ends cleanly.
#include <cuda_bf16.h>

#include <new>

#include "common.cuh"
#include "df.cuh"
#include "mbar.cuh"

namespace afmm {

namespace {

constexpr int TC_SLICES = 6;
constexpr int TC_THREADS = 512;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;  // a completion wait gives up after 1 s

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets
// between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 4 consecutive FP32 columns of TMEM
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float v[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 8 consecutive FP32 columns, the load and its wait
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// e with 2^(e-1) <= m < 2^e for normal m > 0
__device__ __forceinline__ int grid_exp(float m) { return (int)((__float_as_uint(m) >> 23) & 0xff) - 126; }

// 1.5 * 2^(23 + e): (a + c) - c rounds a to a multiple of 2^e (|a| < 2^(e + 22))
__device__ __forceinline__ float round_magic(int e) { return __uint_as_float((uint32_t)(127 + 23 + e) << 23 | 0x400000u); }

// the six digits of v = hi + lo on the grid 2^E > |v|: digit s is a multiple of 2^(E-8-8s)
// with at most 8 significant bits; the digits of hi are exact, lo joins at the fourth digit
// with one FP32 rounding (below 2^(E-48))
template <int NS>
__device__ __forceinline__ void digits(float hi, float lo, int E, float d[NS])
{
    float a = hi;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (s == 3) a = __fadd_rn(a, lo);
        const float c = round_magic(E - 8 - 8 * s);
        const float t = __fsub_rn(__fadd_rn(a, c), c);
        d[s] = t;
        a = __fsub_rn(a, t);
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float x, float y)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<uint32_t *>(&h);
}

// the tables are indexed per lane: read them from shared memory (a kernel parameter lives
// in the constant bank, where divergent indices serialise)
__device__ __forceinline__ void stage_tables(const TcTables &src, TcTables &dst)
{
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(TcTables) / 4); i += blockDim.x) d[i] = s[i];
}

}  // namespace

struct S2LTcArgs {
    const int32_t *unit_box, *unit_col, *s2l, *station_of_col;
    int level, nm, M, nc;
    const float2 *gexp_df;        // [station][16][mode][(M+1)^2 (2M+1)] FP32 pairs
    const __nv_bfloat16 *asl;     // [box][mode][re, im][NS][KP] digit slices of A
    void *loc_re, *loc_im;        // [box][mode][ncoef] of the locals' type, += F
    int *err;                     // set to 1 when a bounded wait runs out
    int inject_timeout;           // test hook: the first slot with work issues no MMA and no commit
};

// ---- A operand: digit slices of j! S_ij per (box, mode, re/im) row, one warp per row
__device__ __forceinline__ dfv to_df(double x) { return df_from_double(x); }
__device__ __forceinline__ dfv to_df(float x) { return df_make(x, 0.f); }
__device__ __forceinline__ dfv to_df(float2 x) { return df_make(x.x, x.y); }

// local += (S + E + v) / l!  (S, E: the exact levels' pair; v: the FP32 levels)
__device__ __forceinline__ void add_local(double &d, float S, float E, float v, float2 rl)
{
    d += (((double)S + (double)E) + (double)v) * ((double)rl.x + (double)rl.y);
}
__device__ __forceinline__ void add_local(float &d, float S, float E, float v, float2 rl)
{
    d += (float)((((double)S + (double)E) + (double)v) * ((double)rl.x + (double)rl.y));
}
__device__ __forceinline__ void add_local(float2 &d, float S, float E, float v, float2 rl)
{
    const dfv f = df_mul(df_add(two_sum(S, E), df_make(v, 0.f)), df_make(rl.x, rl.y));
    const dfv r = df_add(df_make(d.x, d.y), f);
    d = make_float2(r.hi, r.lo);
}

template <int KP, int NS, typename MT>
__global__ void __launch_bounds__(256) k_slice_moments(const MT *__restrict__ mre, const MT *__restrict__ mim,
                                                       int64_t nbox, int nm, int nc, const TcTables tp,
                                                       __nv_bfloat16 *__restrict__ out)
{
    __shared__ TcTables tt;
    stage_tables(tp, tt);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= nbox * nm * 2) return;
    const int reim = (int)(row & 1);
    const int64_t bm = row >> 1;  // box * nm + mode
    const MT *src = (reim ? mim : mre) + bm * nc;
    constexpr int PER = (KP + 31) / 32;
    dfv v[PER];
    float m = 0.f;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int ij = lane + 32 * t;
        v[t] = df_make(0.f, 0.f);
        if (ij < nc) {
            const float2 jf = tt.jfact[tt.cj[ij]];
            v[t] = df_mul(to_df(src[ij]), df_make(jf.x, jf.y));
            m = fmaxf(m, fabsf(v[t].hi));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const bool live = m >= 1e-30f && m < 1e30f;
    const int E = live ? grid_exp(m) + 1 : 0;
    __nv_bfloat16 *dst = out + row * (NS * KP);
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int ij = lane + 32 * t;
        if (ij < KP) {
            float d[NS];
            if (live && ij < nc)
                digits<NS>(v[t].hi, v[t].lo, E, d);
            else
#pragma unroll
                for (int s = 0; s < NS; ++s) d[s] = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) dst[s * KP + ij] = __float2bfloat16_rn(d[s]);
        }
    }
}

// ---- the operator: one block of 16 warps per (unit of up to 64 boxes, mode)
//
// Per slot: stage the slot's Taylor-coefficient cube (FP32 pairs) in shared memory, build the
// six digit slices of B from it (column grids first), then stream the six digit slices of A
// through two buffers while thread 0 issues the 21 slice-pair MMAs per K step, and finally
// drain the four exact levels into the FP32-pair registers.  Thread (warp w, lane) owns TMEM
// lane 32 (w % 4) + lane (box (w % 2) 32 + lane, re/im w % 4 / 2) and a quarter of the columns.
template <int KP, int NS, typename LT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_s2l_tc(const S2LTcArgs a, const TcTables tp)
{
    // NS digit slices (6: FP64 path, 4: MIXED); levels 0 .. NE-1 exact and drained per slot,
    // level NE (and above) in FP32 over all slots
    constexpr int NE = NS == 6 ? 4 : 2;
    constexpr int KG = KP / 8;              // core matrices along K
    constexpr int BT = KP * KP * 2;         // bytes of one B slice (N = KP rows)
    constexpr int AT = 128 * KP * 2;        // bytes of one A slice buffer
    constexpr int QC = KP / 4;              // accumulator columns drained per thread
    constexpr uint32_t IDESC = umma_idesc(128, KP);
    constexpr uint32_t IDESC2 = umma_idesc(128, 2 * KP <= 256 ? 2 * KP : KP);  // two B slices at once
    constexpr int NACC = NE + 1;            // accumulators: the exact levels and the rest
    static_assert(NACC * KP <= 512, "TMEM holds 512 FP32 columns");
    constexpr uint32_t NCOL = NACC * KP <= 32 ? 32 : NACC * KP <= 64 ? 64 : NACC * KP <= 128 ? 128 : NACC * KP <= 256 ? 256 : 512;
    constexpr int NW = TC_THREADS / 32;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *sB = smem;                                       // [NS][KP rows][KP] bf16
    uint8_t *sA = smem + NS * BT;                             // [2][128 rows][KP] bf16
    // the slot's cube [(M+1)^2 (2M+1)]: FP32 pairs, or (128-wide tiles, 4 slices) the high
    // words only, which keeps the block within shared memory
    constexpr bool C32 = KP > 112;
    static_assert(!C32 || NS == 4, "128-wide tiles with 4 digit slices only");
    float2 *sE = reinterpret_cast<float2 *>(sA + 2 * AT);
    float *sE32 = reinterpret_cast<float *>(sA + 2 * AT);
    auto cube = [&](int i) -> float2 {
        if constexpr (C32)
            return make_float2(sE32[i], 0.f);
        else
            return sE[i];
    };
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    __shared__ int bx[64];
    __shared__ long long rbase[128];        // element offset of each A row's slices, or -1
    __shared__ int colE[KP];
    __shared__ int offK[2][KP], offI[2][KP];  // cube offsets (outward, inward) of kl and ij
    __shared__ float2 rj[16];               // 1 / j! as FP32 pairs
    __shared__ int wait_ok;
    __shared__ int sdr[27], sdz[27];        // slot offsets of the unit's parity
    __shared__ int sflag[27], act_ko[27], nact_s;  // active slots, as positions in the order
    __shared__ uint4 fmask[2][KG];          // sign bits of the K chunks: odd j (0), valid ij (1)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t u = blockIdx.x;
    const int n = blockIdx.y;
    const int M = a.M, nc = a.nc, nm = a.nm, W = M + 1, C2 = 2 * M + 1;
    const int slab = W * W * C2;
    if (tid < 64) bx[tid] = a.unit_box[u * 64 + tid];
    // separable cube offsets: outward (k W + i) C2 + j + l, inward (i W + k) C2 + j + l;
    // the low 4 bits carry l (for kl) and j (for ij)
    for (int t = tid; t < KP; t += TC_THREADS) {
        int oo = 0, oi = 0, po = 0, pi = 0;
        if (t < nc) {
            const int x = tp.ci[t], y = tp.cj[t];
            oo = x * W * C2 + y;  // as kl: k W C2 + l
            oi = x * C2 + y;      // as kl (inward): k C2 + l
            po = x * C2 + y;      // as ij: i C2 + j
            pi = x * W * C2 + y;  // as ij (inward): i W C2 + j
        }
        offK[0][t] = oo << 4 | (t < nc ? tp.cj[t] : 0);
        offK[1][t] = oi << 4 | (t < nc ? tp.cj[t] : 0);
        offI[0][t] = po << 4 | (t < nc ? tp.cj[t] : 0);
        offI[1][t] = pi << 4 | (t < nc ? tp.cj[t] : 0);
    }
    if (tid < 16) rj[tid] = tp.rjl[tid * 16];
    const int ucol = a.unit_col[u];
    const int col = ucol & 0xffff, pz = (ucol >> 30) & 1, pr = col & 1;
    // Slots (dr, dz) and (dr, -dz) share the cube, the station and the orientation; their B
    // operands differ by the sign (-1)^(j + l) of each entry (G is even in x), and the digits
    // of -v are the digits of v negated.  So mirrored slots run back to back (tp.ord) and the
    // second takes the first one's B with those signs flipped instead of a new slicing.
    if (tid < 27) {
        s2l_offset(pr, pz, tid, &sdr[tid], &sdz[tid]);
        sflag[tid] = 0;
    }
    for (int kc = tid; kc < KG; kc += TC_THREADS) {
        uint32_t mj[4], mv[4];
        for (int w = 0; w < 4; ++w) {
            mj[w] = mv[w] = 0u;
            for (int h = 0; h < 2; ++h) {
                const int ij = kc * 8 + 2 * w + h;
                if (ij < nc) {
                    mv[w] |= 0x8000u << (16 * h);
                    if (tp.cj[ij] & 1) mj[w] |= 0x8000u << (16 * h);
                }
            }
        }
        fmask[0][kc] = make_uint4(mj[0], mj[1], mj[2], mj[3]);
        fmask[1][kc] = make_uint4(mv[0], mv[1], mv[2], mv[3]);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;  // accumulator lv (0 .. NE) at TMEM columns [lv KP, (lv + 1) KP)

    // thread 0 polls the mbarrier (bounded); the block learns the outcome at the barrier
    uint32_t nphase[2] = {0, 0};
    bool pend[2] = {false, false};
    bool abort_ = false;
    auto wait_buf = [&](int b) {
        if (!pend[b] || abort_) return;
        if (tid == 0) {
            const uint32_t par = (nphase[b] - 1) & 1;
            bool ok = mbar_try(&mbar[b], par);
            const unsigned long long t0 = global_ns();
            while (!ok && global_ns() - t0 < TC_WAIT_NS) ok = mbar_try(&mbar[b], par);
            wait_ok = ok;
            if (!ok) *(volatile int *)a.err = 1;
        }
        __syncthreads();
        pend[b] = false;
        if (!wait_ok) abort_ = true;
    };

    // FP32-pair accumulators of the exact levels: one TMEM lane x QC columns
    const int q = warp & 3;
    const int row = 32 * q + lane, c0 = (warp >> 2) * QC;
    float accS[QC], accE[QC];
#pragma unroll
    for (int t = 0; t < QC; ++t) accS[t] = accE[t] = 0.f;
    bool any_work = false;
    bool lx_init = false;  // thread 0: the inexact accumulator holds a sum

    constexpr int ntaskB = KP * KG;   // 16-byte chunks of one B slice
    constexpr int ntaskA = 128 * KG;  // 16-byte chunks of one A slice
    const int par = pr + 2 * pz;
    // the active slots (some box of the unit has a source box there; the table holds -1 for
    // positions outside the level's square), in processing order
    for (int e = tid; e < 64 * 27; e += TC_THREADS) {
        const int b = bx[e / 27], slot = e % 27;
        if (b >= 0 && a.s2l[(size_t)b * 27 + slot] >= 0) sflag[slot] = 1;
    }
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int ko = 0; ko < 27; ++ko)
            if (sflag[tp.ord[par][ko]]) act_ko[c++] = ko;
        nact_s = c;
    }
    __syncthreads();
    const int nact = nact_s;
    // a slot whose axial mirror ran just before it takes that slot's B with signs flipped
    auto is_mirror = [&](int k) { return k > 0 && tp.mir[par][act_ko[k]] && act_ko[k - 1] == act_ko[k] - 1; };
    // A slice s of the current slot -> buffer b (rows without a source box read zeros)
    auto load_A = [&](int s, int b) {
        uint8_t *dstb = sA + b * AT;
#pragma unroll
        for (int T0 = 0; T0 < ntaskA; T0 += TC_THREADS) {
            const int T = T0 + tid;
            if (T < ntaskA) {
                const int r = (T / (KG * 8)) * 8 + (T & 7), kc = (T >> 3) % KG;
                const long long rb = rbase[r];
                const __nv_bfloat16 *g = rb >= 0 ? a.asl + rb + s * KP + kc * 8 : a.asl;
                cp_async16(dstb + T * 16, g, rb >= 0 ? 16 : 0);
            }
        }
        cp_async_commit();
    };
    // active slot k's A rows, its cube (8-byte copies: the cube's offset is a multiple of 8
    // bytes only; a mirror slot needs none, its group is committed empty) and A slice 0.
    // Issued before the previous slot's drain, which touches no shared memory.
    auto issue_slot = [&](int k) {
        const int slot = tp.ord[par][act_ko[k]];
        if (tid < 128) {
            const int b = bx[tid & 63];
            const int s2 = b >= 0 ? a.s2l[(size_t)b * 27 + slot] : -1;
            rbase[tid] = s2 >= 0 ? (((long long)s2 * nm + n) * 2 + (tid >> 6)) * NS * KP : -1ll;
        }
        __syncthreads();
        if (!is_mirror(k)) {
            const int dr = sdr[slot], dz = sdz[slot];
            const int scol = col + dr;
            const int station = dr < 0 ? scol : col;
            const int sidx = a.station_of_col[station];
            const int ea = dr < 0 ? -dr : dr, eb = dz < 0 ? -dz : dz;
            const float2 *Eg = a.gexp_df + (((size_t)sidx * 16 + ea * 4 + eb) * nm + n) * (size_t)slab;
            for (int t = tid; t < slab; t += TC_THREADS)
                if constexpr (C32)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(sE32 + t)), "l"(&Eg[t].x) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sE + t)), "l"(Eg + t) : "memory");
        }
        cp_async_commit();
        load_A(0, 0);
    };
    if (nact > 0) issue_slot(0);
    for (int k = 0; k < nact && !abort_; ++k) {
        const int slot = tp.ord[par][act_ko[k]];
        const int dr = sdr[slot], dz = sdz[slot];
        const bool first_slot = k == 0;
        any_work = true;
        const int inward = dr > 0 ? 1 : 0;
        const bool backward = dz > 0;
        const bool mirror = is_mirror(k);
        cp_async_wait<1>();  // the cube (A slice 0 may still be in flight)
        __syncthreads();

        if (mirror) {
            // B of the mirror slot with the signs of the entries of odd j + l flipped
            // (zero digits keep their sign, as the slicing would give them)
            constexpr int ntaskF = NS * KP * KG;  // 16-byte chunks of all slices
            for (int T = tid; T < ntaskF; T += TC_THREADS) {
                const int t = T % ntaskB;
                const int kl = (t / (KG * 8)) * 8 + (t & 7), kc = (t >> 3) % KG;
                if (kl >= nc) continue;
                const uint4 mj = fmask[0][kc], mv = fmask[1][kc];
                const bool lodd = (offK[0][kl] & 15) & 1;
                uint4 *q4 = reinterpret_cast<uint4 *>(sB + (T / ntaskB) * BT + t * 16);
                uint4 v = *q4;
                auto fl = [&](uint32_t w, uint32_t j, uint32_t va) {
                    const uint32_t m = lodd ? (j ^ va) : j;                        // odd j + l, valid ij
                    const uint32_t nz = ((w & 0x7fff7fffu) + 0x7fff7fffu) & 0x80008000u;  // nonzero halves
                    return w ^ (m & nz);
                };
                v.x = fl(v.x, mj.x, mv.x);
                v.y = fl(v.y, mj.y, mv.y);
                v.z = fl(v.z, mj.z, mv.z);
                v.w = fl(v.w, mj.w, mv.w);
                *q4 = v;
            }
        } else {
            // B: pass 1, the grid exponent of every column kl (max over ij of |E / j!|)
            for (int kl = warp; kl < KP; kl += NW) {
                float m = 0.f;
                if (kl < nc) {
                    const int ok = offK[inward][kl] >> 4;
                    for (int ij = lane; ij < nc; ij += 32) {
                        const int oi = offI[inward][ij];
                        m = fmaxf(m, fabsf(cube(ok + (oi >> 4)).x) * rj[oi & 15].x);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) colE[kl] = (m >= 1e-30f && m < 1e30f) ? grid_exp(m) + 1 : -1000;
            }
            __syncthreads();
            // B: pass 2, digits of E_{k,i,j+l} / j! into the NS slices (chunk T at byte 16 T)
            for (int T = tid; T < ntaskB; T += TC_THREADS) {
                const int kl = (T / (KG * 8)) * 8 + (T & 7), kc = (T >> 3) % KG;
                uint32_t w[NS][4];
#pragma unroll
                for (int s = 0; s < NS; ++s) w[s][0] = w[s][1] = w[s][2] = w[s][3] = 0u;
                const int Ec = kl < nc ? colE[kl] : -1000;
                if (Ec > -1000) {
                    const int okl = offK[inward][kl];
                    const int ok = okl >> 4, l = okl & 15;
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        float dd[2][NS];
#pragma unroll
                        for (int e1 = 0; e1 < 2; ++e1) {
                            const int ij = kc * 8 + e2 * 2 + e1;
                            if (ij < nc) {
                                const int oi = offI[inward][ij];
                                const int j = oi & 15;
                                float2 ev = cube(ok + (oi >> 4));
                                if (backward && ((j + l) & 1)) ev = make_float2(-ev.x, -ev.y);
                                const float2 rf = rj[j];
                                const dfv v = df_mul(df_make(ev.x, ev.y), df_make(rf.x, rf.y));
                                digits<NS>(v.hi, v.lo, Ec, dd[e1]);
                            } else {
#pragma unroll
                                for (int s = 0; s < NS; ++s) dd[e1][s] = 0.f;
                            }
                        }
#pragma unroll
                        for (int s = 0; s < NS; ++s) w[s][e2] = pack_bf16(dd[0][s], dd[1][s]);
                    }
                }
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    *reinterpret_cast<uint4 *>(sB + s * BT + T * 16) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
            }
        }

        // slices of A in turn, double-buffered; slice i meets B slices 0 .. NS - 1 - i
        for (int i = 0; i < NS; ++i) {
            const int b = i & 1;
            if (i + 1 < NS) {
                wait_buf(b ^ 1);
                if (abort_) break;
                load_A(i + 1, b ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0 && !(a.inject_timeout && first_slot)) {
                tc_fence_after();
                const uint32_t abase = smem_u32(sA + b * AT), bbase = smem_u32(sB);
                // B slices j and j + 1 are adjacent in shared memory and levels lv and lv + 1
                // adjacent in tensor memory: one MMA of N = 2 KP covers both products when the
                // two accumulators take the same accumulate flag (both exact, or the exact level
                // before NE in phases i > 0, where NE already holds a sum)
                for (int j = 0; j + i < NS;) {
                    const int lv = i + j < NE ? i + j : NE;
                    const bool two = 2 * KP <= 256 && j + 1 + i < NS && lv < NE && (lv + 1 < NE || i > 0);
                    for (int ks = 0; ks < KP / 16; ++ks) {
                        const uint64_t ad = umma_desc(abase + ks * 256, 128, KG * 128);
                        const uint64_t bd = umma_desc(bbase + j * BT + ks * 256, 128, KG * 128);
                        // exact levels restart every slot with the pair (0, lv); level NE spans all slots
                        const uint32_t acc = lv < NE ? (ks > 0 || i > 0) : (ks > 0 || lx_init);
                        umma_bf16(tmem + (uint32_t)(KP * lv), ad, bd, two ? IDESC2 : IDESC, acc);
                        if (lv == NE) lx_init = true;
                    }
                    j += two ? 2 : 1;
                }
                umma_commit(&mbar[b]);
            }
            ++nphase[b];
            pend[b] = true;
        }
        if (abort_) break;
        // all MMAs of the slot complete -> drain the exact levels (two-sum into the pair;
        // level 3 is small enough to join the low word with one rounding)
        wait_buf(1);
        wait_buf(0);
        if (abort_) break;
        if (k + 1 < nact) issue_slot(k + 1);  // its copies land during the drain
        tc_fence_after();
#pragma unroll
        for (int lv = 0; lv < NE; ++lv) {
#pragma unroll
            for (int c8 = 0; c8 < QC; c8 += 8) {  // 8 columns per load and wait (4 for a remainder)
            float v[8];
            if (c8 + 8 <= QC)
                tmem_ld8(tmem + (uint32_t)(KP * lv) + ((uint32_t)(32 * q) << 16) + c0 + c8, v);
            else
                tmem_ld4(tmem + (uint32_t)(KP * lv) + ((uint32_t)(32 * q) << 16) + c0 + c8, v);
#pragma unroll
            for (int tt = 0; tt < 8 && c8 + tt < QC; ++tt) {
                const int t = c8 + tt;
                float &S = accS[t], &Er = accE[t];
                if (lv == 3) {
                    Er = __fadd_rn(Er, v[tt]);
                } else {
                    const float s = __fadd_rn(S, v[tt]);
                    const float bb = __fsub_rn(s, S);
                    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(v[tt], bb));
                    Er = __fadd_rn(Er, err);
                    S = s;
                }
            }
            }
        }
        tc_fence_before();
        __syncthreads();
    }

    // the inexact levels (accumulated over all slots), 1 / l!, and the write-back
    if (!abort_ && any_work) {
        tc_fence_after();
        const int bl = row & 63, reim = row >> 6;
        const int box = bx[bl];
        LT *dst = box >= 0 ? static_cast<LT *>(reim ? a.loc_im : a.loc_re) + ((size_t)box * nm + n) * nc : nullptr;
#pragma unroll
        for (int c = 0; c < QC / 4; ++c) {
            float v[4];
            tmem_ld4(tmem + (uint32_t)(NE * KP) + ((uint32_t)(32 * q) << 16) + c0 + 4 * c, v);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int kl = c0 + 4 * c + t;
                if (dst && kl < nc) add_local(dst[kl], accS[4 * c + t], accE[4 * c + t], v[t], rj[offK[0][kl] & 15]);
            }
        }
    }
    cp_async_wait<0>();  // no copy of this block is still in flight
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

// ---- host side
static int tc_kp(int nc) { return (nc + 15) / 16 * 16; }

bool s2l_tc_enabled(afmm_plan p)
{
    // FP64 path: 6 digit slices, five accumulators of KP columns in the 512 TMEM columns
    // and exact FP32 levels (4 KP products of <= 2^15 units below 2^24): KP <= 96 (order
    // <= 12).  MIXED: 4 slices, three accumulators, level 1 below 2^22 units: KP <= 128
    // (order <= 14)
    if (p->opt.s2l_engine != 0) return false;
    if (p->precision == AFMM_FP64) return p->ncoef <= 96;
    return p->precision == AFMM_MIXED && p->ncoef <= 128;
}

// digit slices per operand: six (48 bits) for the FP64 path, four (32 bits) for MIXED (three
// cost 24-bit truncation, 6e-6 on cfg2, above the FP32 near field's 1e-6)
static int tc_slices(afmm_plan p) { return p->precision == AFMM_MIXED ? 4 : TC_SLICES; }

int64_t s2l_tc_slice_elems(afmm_plan p, int64_t nbox)
{
    return nbox * p->nmodes * 2 * tc_slices(p) * (int64_t)tc_kp(p->ncoef);
}

afmm_status make_tc_tables(afmm_plan p)
{
    TcTables *t = new (std::nothrow) TcTables();
    if (!t) return AFMM_ENOMEM;
    double f[16];  // j! (exact in FP64)
    f[0] = 1.0;
    for (int i = 1; i < 16; ++i) f[i] = f[i - 1] * i;
    for (int j = 0; j < 16; ++j) {
        const float fh = (float)f[j];
        t->jfact[j] = make_float2(fh, (float)(f[j] - (double)fh));
        for (int l = 0; l < 16; ++l) {
            double x = 1.0 / (f[j] * f[l]);
            float hi = (float)x;
            t->rjl[j * 16 + l] = make_float2(hi, (float)(x - (double)hi));
        }
    }
    for (int par = 0; par < 4; ++par) {
        bool done[27] = {};
        int c = 0;
        for (int s0 = 0; s0 < 27; ++s0) {
            if (done[s0]) continue;
            int dr0, dz0;
            s2l_offset(par & 1, par >> 1, s0, &dr0, &dz0);
            t->ord[par][c] = (int8_t)s0;
            t->mir[par][c++] = 0;
            done[s0] = true;
            for (int s1 = s0 + 1; s1 < 27 && dz0 != 0; ++s1) {
                int dr1, dz1;
                s2l_offset(par & 1, par >> 1, s1, &dr1, &dz1);
                if (!done[s1] && dr1 == dr0 && dz1 == -dz0) {
                    t->ord[par][c] = (int8_t)s1;
                    t->mir[par][c++] = 1;
                    done[s1] = true;
                    break;
                }
            }
        }
    }
    for (int i = 0; i < 128; ++i) t->ci[i] = t->cj[i] = -1;
    int idx = 0;
    for (int a = 0; a <= p->M; ++a)
        for (int b = 0; a + b <= p->M; ++b, ++idx) {
            t->ci[idx] = (int8_t)a;
            t->cj[idx] = (int8_t)b;
        }
    p->tct = t;
    return AFMM_OK;
}

template <int KP, int NS, typename R>
static afmm_status launch_tc_k(afmm_plan p, int l, const R *mre, const R *mim, R *lre, R *lim)
{
    Level &v = p->lv[l];
    cudaStream_t st = p->stream;
    const int nm = p->nmodes, nc = p->ncoef;
    __nv_bfloat16 *asl = reinterpret_cast<__nv_bfloat16 *>(p->asl);
    const int64_t rows = v.nbox * nm * 2;
    k_slice_moments<KP, NS, R><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(mre, mim, v.nbox, nm, nc,
                                                                                  *p->tct, asl);
    AFMM_LAUNCH_CHECK();
    S2LTcArgs a;
    a.unit_box = v.unit64_box;
    a.unit_col = v.unit64_col;
    a.s2l = v.s2l;
    a.station_of_col = v.station_of_col;
    a.level = l;
    a.nm = nm;
    a.M = p->M;
    a.nc = nc;
    a.gexp_df = p->gexp_df;
    a.asl = asl;
    a.loc_re = lre;
    a.loc_im = lim;
    a.err = p->err_dev;
    a.inject_timeout = p->inject_tc_timeout;
    const int W = p->M + 1;
    const size_t sm = (size_t)NS * KP * KP * 2 + (size_t)2 * 128 * KP * 2 + (size_t)W * W * (2 * p->M + 1) * (KP > 112 ? 4 : 8);
    if (sm > 227 * 1024) return AFMM_EUNSUPPORTED;
    AFMM_CUDA(cudaFuncSetAttribute(k_s2l_tc<KP, NS, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_s2l_tc<KP, NS, R><<<dim3((unsigned)v.nunit64, (unsigned)nm), TC_THREADS, sm, st>>>(a, *p->tct);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

template <int NS, typename R>
static afmm_status launch_tc_ns(afmm_plan p, int l, const R *mre, const R *mim, R *lre, R *lim)
{
    switch (tc_kp(p->ncoef)) {
    case 16: return launch_tc_k<16, NS, R>(p, l, mre, mim, lre, lim);
    case 32: return launch_tc_k<32, NS, R>(p, l, mre, mim, lre, lim);
    case 48: return launch_tc_k<48, NS, R>(p, l, mre, mim, lre, lim);
    case 64: return launch_tc_k<64, NS, R>(p, l, mre, mim, lre, lim);
    case 80: return launch_tc_k<80, NS, R>(p, l, mre, mim, lre, lim);
    case 96: return launch_tc_k<96, NS, R>(p, l, mre, mim, lre, lim);
    }
    if constexpr (NS == 4) {
        if (tc_kp(p->ncoef) == 112) return launch_tc_k<112, NS, R>(p, l, mre, mim, lre, lim);
        if (tc_kp(p->ncoef) == 128) return launch_tc_k<128, NS, R>(p, l, mre, mim, lre, lim);
    }
    return AFMM_EUNSUPPORTED;
}

afmm_status launch_s2l_tc(afmm_plan p, int l, const double *mre, const double *mim, double *lre, double *lim)
{
    if (p->lv[l].nunit64 == 0) return AFMM_OK;
    if (!p->asl || !p->tct || !p->err_dev || !p->gexp_df) return AFMM_EINVAL;
    return launch_tc_ns<TC_SLICES, double>(p, l, mre, mim, lre, lim);
}

afmm_status launch_s2l_tc(afmm_plan p, int l, const float2 *mre, const float2 *mim, float2 *lre, float2 *lim)
{
    if (p->lv[l].nunit64 == 0) return AFMM_OK;
    if (!p->asl || !p->tct || !p->err_dev || !p->gexp_df) return AFMM_EINVAL;
    return launch_tc_ns<TC_SLICES, float2>(p, l, mre, mim, lre, lim);
}

afmm_status launch_s2l_tc(afmm_plan p, int l, const float *mre, const float *mim, float *lre, float *lim)
{
    if (p->lv[l].nunit64 == 0) return AFMM_OK;
    if (!p->asl || !p->tct || !p->err_dev || !p->gexp_df) return AFMM_EINVAL;
    return launch_tc_ns<4, float>(p, l, mre, mim, lre, lim);
}

}  // namespace afmm
