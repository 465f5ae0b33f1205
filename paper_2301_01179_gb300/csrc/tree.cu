// tree.cu -- quadtree over (r, z): the paper's uniform tree (Sec. 2.1; Algorithm 1, first two
// steps) and the adaptive tree (boxes split only where points are dense, with its near lists).
//
// Domain: the square anchored at (min r, min z) over sources and field points with side
// L = max(r extent, z extent) (the paper's square 0 <= r, z <= r_max, moved to the data).
// A point's box at level l is floor((v - v0) * 2^l / L), clamped to 2^l - 1.  Keys are
// computed once at level 16; 2^l / L is a power-of-two multiple of 2^16 / L, so a level-l
// index is exactly the level-16 index shifted right by 16 - l.
// Depth (uniform tree): the smallest d >= 2 whose non-empty source leaves hold at most
// leaf_size sources on average, unless overridden.  Adaptive tree: see build_levels_adaptive.
// All steps are device kernels; the host reads back a handful of counts.
#include "common.cuh"
#include "df.cuh"
#include <cstring>
#include <vector>
#include <algorithm>

namespace afmm {

// ------------------------------------------------------------------------------------
// validation and bounding square
// ------------------------------------------------------------------------------------
__global__ void k_minmax(const double *__restrict__ r1, const double *__restrict__ z1, int64_t n1,
                         const double *__restrict__ r2, const double *__restrict__ z2, int64_t n2,
                         double *__restrict__ part)
{
    double rmin = INFINITY, rmax = -INFINITY, zmin = INFINITY, zmax = -INFINITY, bad = 0.0;
    int64_t n = n1 + n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double r = i < n1 ? r1[i] : r2[i - n1];
        double z = i < n1 ? z1[i] : z2[i - n1];
        if (!(r > 0.0) || !isfinite(r) || !isfinite(z)) {
            bad += 1.0;
            continue;
        }
        rmin = fmin(rmin, r);
        rmax = fmax(rmax, r);
        zmin = fmin(zmin, z);
        zmax = fmax(zmax, z);
    }
    __shared__ double sh[5][32];
    for (int o = 16; o > 0; o >>= 1) {
        rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        zmin = fmin(zmin, __shfl_xor_sync(0xffffffffu, zmin, o));
        zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0) {
        sh[0][w] = rmin; sh[1][w] = rmax; sh[2][w] = zmin; sh[3][w] = zmax; sh[4][w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int k = 1; k < nw; ++k) {
            sh[0][0] = fmin(sh[0][0], sh[0][k]);
            sh[1][0] = fmax(sh[1][0], sh[1][k]);
            sh[2][0] = fmin(sh[2][0], sh[2][k]);
            sh[3][0] = fmax(sh[3][0], sh[3][k]);
            sh[4][0] += sh[4][k];
        }
        for (int k = 0; k < 5; ++k) part[blockIdx.x * 5 + k] = sh[k][0];
    }
}

__global__ void k_minmax_final(const double *__restrict__ part, int nblk, double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double v[5] = {INFINITY, -INFINITY, INFINITY, -INFINITY, 0.0};
    for (int b = 0; b < nblk; ++b) {
        v[0] = fmin(v[0], part[b * 5 + 0]);
        v[1] = fmax(v[1], part[b * 5 + 1]);
        v[2] = fmin(v[2], part[b * 5 + 2]);
        v[3] = fmax(v[3], part[b * 5 + 3]);
        v[4] += part[b * 5 + 4];
    }
    for (int k = 0; k < 5; ++k) out[k] = v[k];
}

// ------------------------------------------------------------------------------------
// keys and sort
// ------------------------------------------------------------------------------------
__device__ inline uint32_t box_coord16(double v, double v0, double s16)
{
    double f = floor((v - v0) * s16);
    if (f < 0.0) f = 0.0;
    if (f > 65535.0) f = 65535.0;
    return (uint32_t)f;
}

__global__ void k_keys(const double *__restrict__ r, const double *__restrict__ z, int64_t n, int64_t npad,
                       double r0, double z0, double s16, unsigned long long *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) {
        out[i] = ~0ull;
        return;
    }
    uint32_t ir = box_coord16(r[i], r0, s16), iz = box_coord16(z[i], z0, s16);
    out[i] = ((unsigned long long)morton_key(ir, iz) << 32) | (unsigned long long)i;
}

// Bitonic sort of 64-bit keys, ascending; npad a power of two >= 2048.
#define BITONIC_TILE 2048
__global__ void k_bitonic_tile(unsigned long long *__restrict__ a, int64_t k_start, int merge_only)
{
    __shared__ unsigned long long s[BITONIC_TILE];
    int64_t base = (int64_t)blockIdx.x * BITONIC_TILE;
    for (int t = threadIdx.x; t < BITONIC_TILE; t += blockDim.x) s[t] = a[base + t];
    __syncthreads();
    int64_t kfirst = merge_only ? k_start : 2;
    int64_t klast = merge_only ? k_start : BITONIC_TILE;
    for (int64_t k = kfirst; k <= klast; k <<= 1) {
        int jstart = (int)((k >> 1) < (BITONIC_TILE >> 1) ? (k >> 1) : (BITONIC_TILE >> 1));
        for (int j = jstart; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < BITONIC_TILE / 2; t += blockDim.x) {
                int i = 2 * j * (t / j) + (t % j);
                int pr = i + j;
                int64_t gi = base + i;
                bool up = (gi & k) == 0;
                unsigned long long x = s[i], y = s[pr];
                if ((x > y) == up) {
                    s[i] = y;
                    s[pr] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < BITONIC_TILE; t += blockDim.x) a[base + t] = s[t];
}

__global__ void k_bitonic_global(unsigned long long *__restrict__ a, int64_t npad, int64_t j, int64_t k)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= npad / 2) return;
    int64_t i = 2 * j * (t / j) + (t % j);
    int64_t pr = i + j;
    bool up = (i & k) == 0;
    unsigned long long x = a[i], y = a[pr];
    if ((x > y) == up) {
        a[i] = y;
        a[pr] = x;
    }
}

static afmm_status bitonic_sort(unsigned long long *a, int64_t npad, cudaStream_t st)
{
    int64_t tiles = npad / BITONIC_TILE;
    k_bitonic_tile<<<(unsigned)tiles, 1024, 0, st>>>(a, 2, 0);
    AFMM_LAUNCH_CHECK();
    for (int64_t k = 2 * BITONIC_TILE; k <= npad; k <<= 1) {
        for (int64_t j = k >> 1; j >= BITONIC_TILE; j >>= 1) {
            int64_t half = npad / 2;
            k_bitonic_global<<<(unsigned)((half + 255) / 256), 256, 0, st>>>(a, npad, j, k);
            AFMM_LAUNCH_CHECK();
        }
        k_bitonic_tile<<<(unsigned)tiles, 1024, 0, st>>>(a, k, 1);
        AFMM_LAUNCH_CHECK();
    }
    return AFMM_OK;
}

static int64_t pow2_at_least(int64_t n)
{
    int64_t p = BITONIC_TILE;
    while (p < n) p <<= 1;
    return p;
}

// ------------------------------------------------------------------------------------
// scans (exclusive, int32 / int64 counts) for stream compaction
// ------------------------------------------------------------------------------------
__global__ void k_scan_block(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             int64_t *__restrict__ bsum)
{
    __shared__ int64_t ws[32];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int ln = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (ln >= o) x += y;
    }
    if (ln == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = ln < (int)(blockDim.x >> 5) ? ws[ln] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (ln >= o) s += y;
        }
        ws[ln] = s;
    }
    __syncthreads();
    int64_t pre = (w > 0 ? ws[w - 1] : 0) + x - v;  // exclusive
    if (i < n) out[i] = pre;
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = pre + v;
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ boff)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

// exclusive scan of in[0..n) into out[0..n); total written to out[n] (out holds n+1).
// tmp must hold >= 2 * ceil(n/1024) + 64 int64.
static afmm_status scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st)
{
    const int B = 1024;
    int64_t nb = (n + B - 1) / B;
    if (nb < 1) nb = 1;
    int64_t *bsum = tmp, *boff = tmp + nb + 1;
    k_scan_block<<<(unsigned)nb, B, 0, st>>>(in, out, n, bsum);
    AFMM_LAUNCH_CHECK();
    if (nb == 1) {
        // total = bsum[0]
        cudaMemcpyAsync(out + n, bsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
        return AFMM_OK;
    }
    AFMM_TRY(scan_excl(bsum, boff, nb, tmp + 2 * nb + 2, st));
    k_scan_add<<<(unsigned)nb, B, 0, st>>>(out, n, boff);
    AFMM_LAUNCH_CHECK();
    cudaMemcpyAsync(out + n, boff + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    return AFMM_OK;
}

// ------------------------------------------------------------------------------------
// per-point outputs of the sort
// ------------------------------------------------------------------------------------
__global__ void k_copy_words(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst, int n)
{
    if ((int)threadIdx.x < n) dst[threadIdx.x] = src[threadIdx.x];
}

// v = a0 + a1 + a2 exactly: a0 is v rounded to FP32, a1 the remainder rounded to FP32 (the
// remainders are exact in FP64), a2 the last few bits
__device__ __forceinline__ void split_f32x3(double v, float &a0, float &a1, float &a2)
{
    a0 = __double2float_rn(v);
    const double r = v - (double)a0;
    a1 = __double2float_rn(r);
    a2 = __double2float_rn(r - (double)a1);
}

__global__ void k_gather_sorted(const unsigned long long *__restrict__ srt, int64_t n, const double *__restrict__ r,
                                const double *__restrict__ z, double *__restrict__ rs, double *__restrict__ zs,
                                float4 *__restrict__ geo, int32_t *__restrict__ perm, uint32_t *__restrict__ key)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long v = srt[i];
    int32_t idx = (int32_t)(v & 0xffffffffull);
    perm[i] = idx;
    key[i] = (uint32_t)(v >> 32);
    rs[i] = r[idx];
    zs[i] = z[idx];
    // exact FP32 triples of the coordinates and 1 / r as an FP32 pair, for the FP32-pair near
    // field (its coordinate differences then need no FP64 arithmetic)
    float r0, r1, r2, z0, z1, z2;
    split_f32x3(r[idx], r0, r1, r2);
    split_f32x3(z[idx], z0, z1, z2);
    const dfv d = df_from_double(1.0 / r[idx]);
    geo[2 * i] = make_float4(r0, r1, z0, z1);
    geo[2 * i + 1] = make_float4(r2, z2, d.hi, d.lo);
}

// number of distinct level-l prefixes among sorted level-16 keys, l = 2..16
__global__ void k_depth_counts(const uint32_t *__restrict__ key, int64_t n, unsigned long long *__restrict__ cnt)
{
    __shared__ unsigned int c[17];
    if (threadIdx.x < 17) c[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        for (int l = 2; l <= 16; ++l) {
            int sh = 2 * (16 - l);
            if (i == 0 || (key[i] >> sh) != (key[i - 1] >> sh)) atomicAdd(&c[l], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 17 && c[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], (unsigned long long)c[threadIdx.x]);
}

// leaf keys of both point sets, packed for a union sort (key << 32)
__global__ void k_leaf_union(const uint32_t *__restrict__ ks, int64_t ns, const uint32_t *__restrict__ kt, int64_t nf,
                             int sh, int64_t npad, unsigned long long *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    unsigned long long v = ~0ull;
    if (i < ns)
        v = (unsigned long long)(ks[i] >> sh) << 32;
    else if (i < ns + nf)
        v = (unsigned long long)(kt[i - ns] >> sh) << 32;
    out[i] = v;
}

// flags[i] = 1 where a new distinct key starts (keys from a sorted 64-bit array, value >> 32,
// further shifted right by `extra` bits); invalid (~0) entries get 0
__global__ void k_unique_flags(const unsigned long long *__restrict__ a, int64_t n, int extra, int64_t *__restrict__ f)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long v = a[i];
    if (v == ~0ull) {
        f[i] = 0;
        return;
    }
    uint32_t k = (uint32_t)(v >> 32) >> extra;
    f[i] = (i == 0 || ((uint32_t)(a[i - 1] >> 32) >> extra) != k) ? 1 : 0;
}

__global__ void k_unique_scatter(const unsigned long long *__restrict__ a, int64_t n, int extra,
                                 const int64_t *__restrict__ f, const int64_t *__restrict__ pos,
                                 uint32_t *__restrict__ keys)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (f[i]) keys[pos[i]] = (uint32_t)(a[i] >> 32) >> extra;
}

// keys of level l-1 from keys of level l (>> 2), written into a 64-bit array for uniq
__global__ void k_parent_keys(const uint32_t *__restrict__ k, int64_t n, unsigned long long *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (unsigned long long)(k[i] >> 2) << 32;
}

__device__ inline int64_t lower_bound_u32(const uint32_t *__restrict__ a, int64_t n, unsigned long long v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((unsigned long long)a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ inline int64_t find_key(const uint32_t *__restrict__ a, int64_t n, uint32_t v)
{
    int64_t i = lower_bound_u32(a, n, v);
    return (i < n && a[i] == v) ? i : -1;
}

__global__ void k_box_ranges(const uint32_t *__restrict__ bkey, int64_t nbox, int sh, const uint32_t *__restrict__ sk,
                             int64_t ns, const uint32_t *__restrict__ tk, int64_t nf, int2 *__restrict__ srng,
                             int2 *__restrict__ trng)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    unsigned long long lo = (unsigned long long)bkey[b] << sh, hi = ((unsigned long long)bkey[b] + 1) << sh;
    srng[b] = make_int2((int)lower_bound_u32(sk, ns, lo), (int)lower_bound_u32(sk, ns, hi));
    trng[b] = make_int2((int)lower_bound_u32(tk, nf, lo), (int)lower_bound_u32(tk, nf, hi));
}

__global__ void k_parents(const uint32_t *__restrict__ bkey, int64_t nbox, const uint32_t *__restrict__ pkey,
                          int64_t npbox, int32_t *__restrict__ parent)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    parent[b] = (int32_t)find_key(pkey, npbox, bkey[b] >> 2);
}

__global__ void k_child_ranges(const int32_t *__restrict__ parent, int64_t nbox, int2 *__restrict__ child)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int32_t p = parent[b];
    if (b == 0 || parent[b - 1] != p) child[p].x = (int)b;
    if (b == nbox - 1 || parent[b + 1] != p) child[p].y = (int)(b + 1);
}

__global__ void k_s2l_table(const uint32_t *__restrict__ bkey, int64_t nbox, int level, int32_t *__restrict__ tab)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nbox * 27) return;
    int64_t b = t / 27;
    int slot = (int)(t % 27);
    uint32_t k = bkey[b];
    int ti = (int)morton_ir(k), tj = (int)morton_iz(k);
    int dr, dz;
    s2l_offset(ti & 1, tj & 1, slot, &dr, &dz);
    int si = ti + dr, sj = tj + dz, nl = 1 << level;
    int32_t v = -1;
    if (si >= 0 && sj >= 0 && si < nl && sj < nl) v = (int32_t)find_key(bkey, nbox, morton_key(si, sj));
    tab[t] = v;
}

__global__ void k_nbr_table(const uint32_t *__restrict__ bkey, int64_t nbox, int level, int32_t *__restrict__ tab)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nbox * 9) return;
    int64_t b = t / 9;
    int slot = (int)(t % 9);
    uint32_t k = bkey[b];
    int ti = (int)morton_ir(k) + slot / 3 - 1, tj = (int)morton_iz(k) + slot % 3 - 1, nl = 1 << level;
    int32_t v = -1;
    if (ti >= 0 && tj >= 0 && ti < nl && tj < nl) v = (int32_t)find_key(bkey, nbox, morton_key(ti, tj));
    tab[t] = v;
}

__global__ void k_station_flags(const uint32_t *__restrict__ bkey, int64_t nbox, int32_t *__restrict__ flag)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nbox) flag[morton_ir(bkey[b])] = 1;
}

__global__ void k_station_map(const int32_t *__restrict__ flag, int ncol, const int64_t *__restrict__ pos,
                              int32_t *__restrict__ st_of_col, int32_t *__restrict__ col_of_st)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    if (flag[c]) {
        st_of_col[c] = (int32_t)pos[c];
        col_of_st[pos[c]] = c;
    } else {
        st_of_col[c] = -1;
    }
}

__global__ void k_i32_to_i64(const int32_t *__restrict__ a, int64_t n, int64_t *__restrict__ b)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// S2L units: boxes sorted by (column, axial parity, axial index); groups of us (32 for the
// CUDA-core operators, 64 for the tensor-core operator)
__global__ void k_unit_keys(const uint32_t *__restrict__ bkey, int64_t nbox, int64_t npad,
                            unsigned long long *__restrict__ out)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= npad) return;
    if (b >= nbox) {
        out[b] = ~0ull;
        return;
    }
    uint32_t k = bkey[b];
    unsigned long long ir = morton_ir(k), iz = morton_iz(k);
    out[b] = (ir << 48) | ((iz & 1ull) << 47) | (iz << 24) | (unsigned long long)b;
}

__device__ inline unsigned long long unit_group(unsigned long long v) { return v >> 47; }

__global__ void k_unit_flags(const unsigned long long *__restrict__ u, int64_t nbox, int us, int64_t *__restrict__ f)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nbox) return;
    unsigned long long g = unit_group(u[i]);
    int64_t lo = 0, hi = i;  // first index with the same group
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (unit_group(u[mid]) < g)
            lo = mid + 1;
        else
            hi = mid;
    }
    f[i] = ((i - lo) % us == 0) ? 1 : 0;
}

__global__ void k_unit_fill(const unsigned long long *__restrict__ u, int64_t nbox, int us,
                            const int64_t *__restrict__ pos, int32_t *__restrict__ ubox, int32_t *__restrict__ ucol)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nbox) return;
    unsigned long long v = u[i], g = unit_group(v);
    int64_t lo = 0, hi = i;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (unit_group(u[mid]) < g)
            lo = mid + 1;
        else
            hi = mid;
    }
    int64_t rank = i - lo;
    int64_t unit = pos[i - (rank % us)];
    ubox[unit * us + rank % us] = (int32_t)(v & 0xffffffull);
    if (rank % us == 0) ucol[unit] = (int32_t)((v >> 48) | ((v >> 47 & 1ull) << 30));
}

// near-field units: ceil(count/32) per leaf box with field-role points
__global__ void k_near_counts(const int2 *__restrict__ rng, int64_t nbox, int64_t *__restrict__ cnt)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nbox) cnt[b] = (rng[b].y - rng[b].x + 31) / 32;
}

__global__ void k_near_fill(const int2 *__restrict__ rng, int64_t nbox, int level, const int64_t *__restrict__ pos,
                            NearUnit *__restrict__ u)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int64_t p = pos[b];
    for (int s = rng[b].x; s < rng[b].y; s += 32) {
        NearUnit x;
        x.box = (int32_t)b;
        x.begin = s;
        x.end = min(s + 32, rng[b].y);
        x.level = level;
        u[p++] = x;
    }
}

// statistics: near-field pairs and S2L applications
__global__ void k_near_pairs(const int2 *__restrict__ trng, const int2 *__restrict__ srng, const int32_t *__restrict__ nbr,
                             int64_t nbox, unsigned long long *__restrict__ acc)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    long long nt = trng[b].y - trng[b].x, s = 0;
    for (int k = 0; k < 9; ++k) {
        int32_t q = nbr[b * 9 + k];
        if (q >= 0) s += srng[q].y - srng[q].x;
    }
    atomicAdd(acc, (unsigned long long)(nt * s));
    if (nt > 0) atomicMax(acc + 3, (unsigned long long)s);
}

// S2L applications of a level (acc[0]) and the (field point, source) pairs they cover (acc[1])
__global__ void k_s2l_count(const int32_t *__restrict__ tab, const int2 *__restrict__ trng,
                            const int2 *__restrict__ srng, int64_t nbox, unsigned long long *__restrict__ acc)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    unsigned long long s = 0, pp = 0;
    const unsigned long long nt = (unsigned long long)(trng[b].y - trng[b].x);
    for (int k = 0; k < 27; ++k) {
        int32_t q = tab[b * 27 + k];
        if (q >= 0) {
            s += 1;
            pp += nt * (unsigned long long)(srng[q].y - srng[q].x);
        }
    }
    atomicAdd(acc, s);
    atomicAdd(acc + 1, pp);
}

// ------------------------------------------------------------------------------------
// adaptive tree: levels built top-down.  Level 2 holds every non-empty box; a box of level
// l < lmax is split while it holds more than leaf_size sources or field points, or (balance
// rule) while a same-level neighbour holds more than lim = K leaf_size of either, and its
// non-empty children form level l + 1 (sorted by key, since the parents are and the child
// quadrant c = (radial bit << 1) | axial bit is the key's lowest digit).
// ------------------------------------------------------------------------------------
// split flags of level l: more than leaf points of either role, or (balance lim > 0) a
// same-level neighbour with more than lim points of either role
__global__ void k_split_flags(const uint32_t *__restrict__ key, const int2 *__restrict__ srng,
                              const int2 *__restrict__ trng, int64_t nbox, int l, int leaf, int64_t lim,
                              int64_t *__restrict__ flag)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    bool split = srng[b].y - srng[b].x > leaf || trng[b].y - trng[b].x > leaf;
    if (!split && lim > 0) {
        const uint32_t k = key[b];
        const int ir = (int)morton_ir(k), iz = (int)morton_iz(k), nl = 1 << l;
        for (int dr = -1; dr <= 1 && !split; ++dr)
            for (int dz = -1; dz <= 1; ++dz) {
                const int i = ir + dr, j = iz + dz;
                if ((dr == 0 && dz == 0) || i < 0 || j < 0 || i >= nl || j >= nl) continue;
                const int64_t q = find_key(key, nbox, morton_key(i, j));
                if (q >= 0 && (srng[q].y - srng[q].x > lim || trng[q].y - trng[q].x > lim)) {
                    split = true;
                    break;
                }
            }
    }
    flag[b] = split ? 1 : 0;
}

// four candidates per split parent (pkey == nullptr: the 4 boxes of level 1, all split);
// each gets its key, parent and point ranges at level lc, and ne = 1 if it holds a point
__global__ void k_child_cand(const uint32_t *__restrict__ pkey, const int64_t *__restrict__ flag,
                             const int64_t *__restrict__ pos, int64_t npar, int lc, const uint32_t *__restrict__ sk,
                             int64_t ns, const uint32_t *__restrict__ tk, int64_t nf, uint32_t *__restrict__ ckey,
                             int32_t *__restrict__ cpar, int2 *__restrict__ csr, int2 *__restrict__ ctr,
                             int64_t *__restrict__ ne)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 4 * npar) return;
    const int64_t b = t >> 2;
    const uint32_t c = (uint32_t)(t & 3);
    if (pkey && !flag[b]) return;
    const int64_t i = 4 * (pkey ? pos[b] : b) + c;
    const uint32_t k = ((pkey ? pkey[b] : (uint32_t)b) << 2) | c;
    const int sh = 2 * (16 - lc);
    const unsigned long long lo = (unsigned long long)k << sh, hi = ((unsigned long long)k + 1) << sh;
    const int2 rs = make_int2((int)lower_bound_u32(sk, ns, lo), (int)lower_bound_u32(sk, ns, hi));
    const int2 rt = make_int2((int)lower_bound_u32(tk, nf, lo), (int)lower_bound_u32(tk, nf, hi));
    ckey[i] = k;
    cpar[i] = (int32_t)b;
    csr[i] = rs;
    ctr[i] = rt;
    ne[i] = (rs.y > rs.x || rt.y > rt.x) ? 1 : 0;
}

__global__ void k_child_compact(const uint32_t *__restrict__ ckey, const int32_t *__restrict__ cpar,
                                const int2 *__restrict__ csr, const int2 *__restrict__ ctr,
                                const int64_t *__restrict__ ne, const int64_t *__restrict__ pos, int64_t ncand,
                                uint32_t *__restrict__ key, int32_t *__restrict__ par, int2 *__restrict__ srng,
                                int2 *__restrict__ trng)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ncand || !ne[i]) return;
    const int64_t o = pos[i];
    key[o] = ckey[i];
    if (par) par[o] = cpar[i];
    srng[o] = csr[i];
    trng[o] = ctr[i];
}

// leaf ranges for the P2M (empty for split boxes) and the leaf count of a level
__global__ void k_leaf_ranges(const int2 *__restrict__ child, const int2 *__restrict__ srng,
                              const int2 *__restrict__ trng, int64_t nbox, int2 *__restrict__ sl,
                              int2 *__restrict__ tl, unsigned long long *__restrict__ nleaf)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const bool leaf = child[b].x >= child[b].y;
    sl[b] = leaf ? srng[b] : make_int2(0, 0);
    tl[b] = leaf ? trng[b] : make_int2(0, 0);
    if (leaf) atomicAdd(nleaf, 1ull);
}

// per-level tables of the adaptive tree, passed by value
struct AdTab {
    const uint32_t *key[AFMM_MAX_LEVEL + 1];
    const int2 *child[AFMM_MAX_LEVEL + 1];
    const int2 *srng[AFMM_MAX_LEVEL + 1];
    const int2 *trng[AFMM_MAX_LEVEL + 1];
    int64_t nbox[AFMM_MAX_LEVEL + 1];
};

// The near list of leaf b of level l: (a) the existing boxes of level l in the 3 x 3 block
// around b (b included; a split box brings its whole subtree), (b) for every coarser level
// c >= 2, the leaves of level c among the 8 boxes around b's ancestor.  A source leaf C and a
// field leaf B are summed directly exactly when their ancestors at the coarser of their two
// levels touch; every other pair meets in the interaction list of the first level at which
// their ancestors separate.  f(level, box) is called once per listed box.
template <typename F>
__device__ void anear_visit(const AdTab &T, int l, int64_t b, F f)
{
    const uint32_t k = T.key[l][b];
    const int ir = (int)morton_ir(k), iz = (int)morton_iz(k);
    for (int dr = -1; dr <= 1; ++dr)
        for (int dz = -1; dz <= 1; ++dz) {
            const int i = ir + dr, j = iz + dz, nl = 1 << l;
            if (i < 0 || j < 0 || i >= nl || j >= nl) continue;
            const int64_t q = find_key(T.key[l], T.nbox[l], morton_key(i, j));
            if (q >= 0) f(l, q);
        }
    for (int c = l - 1; c >= 2; --c) {
        const int ai = ir >> (l - c), aj = iz >> (l - c), nc = 1 << c;
        for (int dr = -1; dr <= 1; ++dr)
            for (int dz = -1; dz <= 1; ++dz) {
                const int i = ai + dr, j = aj + dz;
                if ((dr == 0 && dz == 0) || i < 0 || j < 0 || i >= nc || j >= nc) continue;
                const int64_t q = find_key(T.key[c], T.nbox[c], morton_key(i, j));
                if (q >= 0 && T.child[c][q].x >= T.child[c][q].y) f(c, q);
            }
    }
}

__global__ void k_anear_count(const AdTab T, int l, int64_t *__restrict__ cnt, unsigned long long *__restrict__ mx)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= T.nbox[l]) return;
    int n = 0;
    if (T.child[l][b].x >= T.child[l][b].y) anear_visit(T, l, b, [&](int, int64_t) { ++n; });
    cnt[b] = n;
    atomicMax(mx, (unsigned long long)n);
}

// ranges of both roles; acc[0] += (field points) x (listed sources), acc[1] the transposed
__global__ void k_anear_fill(const AdTab T, int l, const int64_t *__restrict__ off, int2 *__restrict__ rs,
                             int2 *__restrict__ rt, unsigned long long *__restrict__ acc)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= T.nbox[l] || T.child[l][b].x < T.child[l][b].y) return;
    int64_t o = off[b];
    unsigned long long ss = 0, st = 0;
    anear_visit(T, l, b, [&](int c, int64_t q) {
        const int2 a = T.srng[c][q], z = T.trng[c][q];
        rs[o] = a;
        rt[o] = z;
        ++o;
        ss += (unsigned long long)(a.y - a.x);
        st += (unsigned long long)(z.y - z.x);
    });
    const int2 mb = T.trng[l][b], ms = T.srng[l][b];
    atomicAdd(acc, (unsigned long long)(mb.y - mb.x) * ss);
    atomicAdd(acc + 1, (unsigned long long)(ms.y - ms.x) * st);
    if (mb.y > mb.x) atomicMax(acc + 3, ss);  // the largest direct sum of a leaf with field points
}

// near-field units of the adaptive tree: ceil(count / 32) per leaf with points of the role
__global__ void k_anear_units_count(const int2 *__restrict__ rng, const int2 *__restrict__ child, int64_t nbox,
                                    int64_t *__restrict__ cnt)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    cnt[b] = child[b].x >= child[b].y ? (rng[b].y - rng[b].x + 31) / 32 : 0;
}

__global__ void k_anear_units_fill(const int2 *__restrict__ rng, const int2 *__restrict__ child, int64_t nbox, int l,
                                   const int64_t *__restrict__ pos, NearUnit *__restrict__ u)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox || child[b].x < child[b].y) return;
    int64_t p = pos[b];
    for (int s = rng[b].x; s < rng[b].y; s += 32) {
        NearUnit x;
        x.box = (int32_t)b;
        x.begin = s;
        x.end = min(s + 32, rng[b].y);
        x.level = l;
        u[p++] = x;
    }
}

static inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b > 0 ? (n + b - 1) / b : 1); }

afmm_status readback(afmm_plan p, void *host, const void *dev, size_t bytes)
{
    const int n = (int)(bytes / 8);
    if (bytes % 8 != 0 || n > RB_WORDS || !p->rb_dev) return AFMM_EINVAL;
    k_copy_words<<<1, 32, 0, p->stream>>>((const unsigned long long *)dev, p->rb_dev, n);
    AFMM_LAUNCH_CHECK();
    AFMM_CUDA(cudaStreamSynchronize(p->stream));
    memcpy(host, (const void *)p->rb_host, bytes);
    return AFMM_OK;
}

// compaction helper: distinct keys of a sorted 64-bit array (value >> 32 >> extra) -> keys
static afmm_status uniq_keys(afmm_plan p, const unsigned long long *a, int64_t n, int extra, int64_t *f,
                             int64_t *pos, int64_t *tmp, uint32_t **keys_out, int64_t *count)
{
    cudaStream_t st = p->stream;
    k_unique_flags<<<nblk(n), 256, 0, st>>>(a, n, extra, f);
    AFMM_LAUNCH_CHECK();
    AFMM_TRY(scan_excl(f, pos, n, tmp, st));
    int64_t c = 0;
    AFMM_TRY(readback(p, &c, pos + n, sizeof(int64_t)));
    uint32_t *k = nullptr;
    AFMM_TRY(dalloc_t(p, &k, c > 0 ? c : 1));
    k_unique_scatter<<<nblk(n), 256, 0, st>>>(a, n, extra, f, pos, k);
    AFMM_LAUNCH_CHECK();
    *keys_out = k;
    *count = c;
    return AFMM_OK;
}

// Levels 2..d of the adaptive tree (keys, point ranges, parents, child ranges, leaf ranges)
static afmm_status build_levels_adaptive(afmm_plan p)
{
    cudaStream_t st = p->stream;
    const int64_t ns = p->ns, nf = p->nf;
    const int lmax = p->opt.depth_override > 0 ? p->opt.depth_override : AFMM_MAX_LEVEL;
    const int leaf = p->opt.leaf_size;
    const int64_t lim = p->opt.balance < 0 ? 0 : (int64_t)(p->opt.balance == 0 ? 4 : p->opt.balance) * leaf;
    // boxes of one level are disjoint and non-empty (at most ns + nf); four candidates per
    // split box, in buffers that grow (doubling) with the largest level met so far
    const int64_t bcap = ns + nf + 64;
    int64_t ccap = 0;
    uint32_t *ckey = nullptr;
    int32_t *cpar = nullptr;
    int2 *csr = nullptr, *ctr = nullptr;
    int64_t *ne = nullptr, *cpos = nullptr, *ctmp = nullptr, *flag = nullptr, *fpos = nullptr;
    AFMM_TRY(dalloc_t(p, &flag, bcap));
    AFMM_TRY(dalloc_t(p, &fpos, bcap + 1));
    AFMM_TRY(dalloc_t(p, &ctmp, 2 * (4 * bcap / 1024 + 64) + 256));
    const uint32_t *pkey = nullptr;  // level 1: the four boxes, all split
    int64_t npar = 4;
    int l = 1;
    for (;;) {
        int64_t nsplit = 4;
        if (pkey) {
            if (l >= lmax) break;
            k_split_flags<<<nblk(npar), 256, 0, st>>>(p->lv[l].key, p->lv[l].srng, p->lv[l].trng, npar, l, leaf,
                                                      lim, flag);
            AFMM_LAUNCH_CHECK();
            AFMM_TRY(scan_excl(flag, fpos, npar, ctmp, st));
            AFMM_TRY(readback(p, &nsplit, fpos + npar, sizeof(int64_t)));
            if (nsplit == 0) break;
        }
        const int lc = l + 1;
        const int64_t ncand = 4 * nsplit;
        if (ncand > ccap) {
            ccap = ccap * 2 > ncand ? ccap * 2 : ncand + 64;
            AFMM_TRY(dalloc_t(p, &ckey, ccap));
            AFMM_TRY(dalloc_t(p, &cpar, ccap));
            AFMM_TRY(dalloc_t(p, &csr, ccap));
            AFMM_TRY(dalloc_t(p, &ctr, ccap));
            AFMM_TRY(dalloc_t(p, &ne, ccap));
            AFMM_TRY(dalloc_t(p, &cpos, ccap + 1));
        }
        k_child_cand<<<nblk(4 * npar), 256, 0, st>>>(pkey, flag, fpos, npar, lc, p->s_key, ns, p->t_key, nf, ckey,
                                                      cpar, csr, ctr, ne);
        AFMM_LAUNCH_CHECK();
        AFMM_TRY(scan_excl(ne, cpos, ncand, ctmp, st));
        int64_t nb = 0;
        AFMM_TRY(readback(p, &nb, cpos + ncand, sizeof(int64_t)));
        Level &v = p->lv[lc];
        v.nbox = nb;
        AFMM_TRY(dalloc_t(p, &v.key, nb));
        AFMM_TRY(dalloc_t(p, &v.srng, nb));
        AFMM_TRY(dalloc_t(p, &v.trng, nb));
        if (lc >= 3) AFMM_TRY(dalloc_t(p, &v.parent, nb));
        AFMM_TRY(dalloc_t(p, &v.child, nb));
        AFMM_CUDA(cudaMemsetAsync(v.child, 0, nb * sizeof(int2), st));
        k_child_compact<<<nblk(ncand), 256, 0, st>>>(ckey, cpar, csr, ctr, ne, cpos, ncand, v.key,
                                                     lc >= 3 ? v.parent : nullptr, v.srng, v.trng);
        AFMM_LAUNCH_CHECK();
        if (pkey) {
            k_child_ranges<<<nblk(nb), 256, 0, st>>>(v.parent, nb, p->lv[l].child);
            AFMM_LAUNCH_CHECK();
        }
        pkey = v.key;
        npar = nb;
        l = lc;
    }
    p->d = l;
    unsigned long long *cnt = nullptr;
    AFMM_TRY(dalloc_t(p, &cnt, AFMM_MAX_LEVEL + 1));
    AFMM_CUDA(cudaMemsetAsync(cnt, 0, (AFMM_MAX_LEVEL + 1) * sizeof(unsigned long long), st));
    for (int k = 2; k <= p->d; ++k) {
        Level &v = p->lv[k];
        AFMM_TRY(dalloc_t(p, &v.srng_leaf, v.nbox));
        AFMM_TRY(dalloc_t(p, &v.trng_leaf, v.nbox));
        k_leaf_ranges<<<nblk(v.nbox), 256, 0, st>>>(v.child, v.srng, v.trng, v.nbox, v.srng_leaf, v.trng_leaf, cnt + k);
        AFMM_LAUNCH_CHECK();
    }
    unsigned long long h[AFMM_MAX_LEVEL + 1];
    AFMM_TRY(readback(p, h, cnt, sizeof(h)));
    for (int k = 2; k <= p->d; ++k) p->lv[k].nleaf = (int64_t)h[k];
    return AFMM_OK;
}

// Near lists (CSR of point ranges per box of every level) and near-field units of the
// adaptive tree; near_pairs counts the (field point, source) pairs summed directly
static afmm_status build_near_adaptive(afmm_plan p)
{
    cudaStream_t st = p->stream;
    const int d = p->d;
    AdTab T;
    memset(&T, 0, sizeof(T));
    int64_t tot = 0;
    for (int l = 2; l <= d; ++l) {
        const Level &v = p->lv[l];
        T.key[l] = v.key;
        T.child[l] = v.child;
        T.srng[l] = v.srng;
        T.trng[l] = v.trng;
        T.nbox[l] = v.nbox;
        p->nl_base[l] = tot;
        tot += v.nbox;
    }
    p->nl_base[d + 1] = tot;
    int64_t *cnt = nullptr, *tmp = nullptr, *upos = nullptr;
    unsigned long long *acc = nullptr;
    AFMM_TRY(dalloc_t(p, &cnt, tot + 1));
    AFMM_TRY(dalloc_t(p, &upos, tot + 1));
    AFMM_TRY(dalloc_t(p, &p->nl_off, tot + 1));
    AFMM_TRY(dalloc_t(p, &tmp, 2 * (tot / 1024 + 64) + 256));
    AFMM_TRY(dalloc_t(p, &acc, 4));
    AFMM_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long), st));
    for (int l = 2; l <= d; ++l) {
        k_anear_count<<<nblk(T.nbox[l]), 256, 0, st>>>(T, l, cnt + p->nl_base[l], acc + 2);
        AFMM_LAUNCH_CHECK();
    }
    AFMM_TRY(scan_excl(cnt, p->nl_off, tot, tmp, st));
    int64_t h2[2] = {0, 0};
    AFMM_TRY(readback(p, &h2[0], p->nl_off + tot, sizeof(int64_t)));
    AFMM_TRY(readback(p, &h2[1], acc + 2, sizeof(int64_t)));
    const int64_t nrg = h2[0];
    p->nl_maxrg = (int)h2[1];
    if (p->nl_maxrg > AFMM_NEAR_MAXRG) return AFMM_EUNSUPPORTED;
    AFMM_TRY(dalloc_t(p, &p->nl_rng[0], nrg > 0 ? nrg : 1));
    AFMM_TRY(dalloc_t(p, &p->nl_rng[1], nrg > 0 ? nrg : 1));
    for (int l = 2; l <= d; ++l) {
        k_anear_fill<<<nblk(T.nbox[l]), 256, 0, st>>>(T, l, p->nl_off + p->nl_base[l], p->nl_rng[0], p->nl_rng[1], acc);
        AFMM_LAUNCH_CHECK();
    }
    for (int dir = 0; dir < 2; ++dir) {
        for (int l = 2; l <= d; ++l) {
            const Level &v = p->lv[l];
            k_anear_units_count<<<nblk(v.nbox), 256, 0, st>>>(dir == 0 ? v.trng : v.srng, v.child, v.nbox,
                                                              cnt + p->nl_base[l]);
            AFMM_LAUNCH_CHECK();
        }
        AFMM_TRY(scan_excl(cnt, upos, tot, tmp, st));
        int64_t nu = 0;
        AFMM_TRY(readback(p, &nu, upos + tot, sizeof(int64_t)));
        p->n_near_unit[dir] = nu;
        AFMM_TRY(dalloc_t(p, &p->near_unit[dir], nu > 0 ? nu : 1));
        for (int l = 2; l <= d; ++l) {
            const Level &v = p->lv[l];
            k_anear_units_fill<<<nblk(v.nbox), 256, 0, st>>>(dir == 0 ? v.trng : v.srng, v.child, v.nbox, l,
                                                             upos + p->nl_base[l], p->near_unit[dir]);
            AFMM_LAUNCH_CHECK();
        }
    }
    unsigned long long h[4];
    AFMM_TRY(readback(p, h, acc, sizeof(h)));
    p->near_pairs = (int64_t)h[0];
    p->near_max_src = (int64_t)h[3];
    return AFMM_OK;
}

afmm_status build_tree(afmm_plan p, const double *src_r, const double *src_z, const double *tgt_r,
                       const double *tgt_z)
{
    cudaStream_t st = p->stream;
    const int64_t ns = p->ns, nf = p->nf;
    // ---- validation and bounding square
    const int mmb = 304;
    double *part = nullptr, *mm = nullptr;
    AFMM_TRY(dalloc_t(p, &part, mmb * 5 + 8));
    mm = part + mmb * 5;
    k_minmax<<<mmb, 256, 0, st>>>(src_r, src_z, ns, tgt_r, tgt_z, nf, part);
    AFMM_LAUNCH_CHECK();
    k_minmax_final<<<1, 32, 0, st>>>(part, mmb, mm);
    AFMM_LAUNCH_CHECK();
    double h_mm[5];
    AFMM_TRY(readback(p, h_mm, mm, sizeof(h_mm)));
    if (h_mm[4] != 0.0) return AFMM_EINVAL;
    p->r0 = h_mm[0];
    p->z0 = h_mm[2];
    double L = fmax(h_mm[1] - h_mm[0], h_mm[3] - h_mm[2]);
    if (!(L > 0.0)) L = 1.0;
    p->L = L;
    const double s16 = 65536.0 / L;

    // ---- keys and sorts
    int64_t nmax = ns > nf ? ns : nf;
    int64_t npad_max = pow2_at_least(ns + nf);
    unsigned long long *srt = nullptr;
    AFMM_TRY(dalloc_t(p, &srt, npad_max));
    int64_t *f = nullptr, *pos = nullptr, *tmp = nullptr;
    // flags/scans run over points, boxes and the 2^l columns of a level (l <= 16)
    int64_t nflag = (npad_max > 65536 ? npad_max : 65536) + 64;
    AFMM_TRY(dalloc_t(p, &f, nflag));
    AFMM_TRY(dalloc_t(p, &pos, nflag + 1));
    AFMM_TRY(dalloc_t(p, &tmp, 2 * (nflag / 1024 + 64) + 256));
    AFMM_TRY(dalloc_t(p, &p->s_r, ns));
    AFMM_TRY(dalloc_t(p, &p->s_z, ns));
    AFMM_TRY(dalloc_t(p, &p->s_perm, ns));
    AFMM_TRY(dalloc_t(p, &p->s_key, ns));
    AFMM_TRY(dalloc_t(p, &p->t_r, nf));
    AFMM_TRY(dalloc_t(p, &p->t_z, nf));
    AFMM_TRY(dalloc_t(p, &p->t_perm, nf));
    AFMM_TRY(dalloc_t(p, &p->t_key, nf));
    AFMM_TRY(dalloc_t(p, &p->s_geo, 2 * ns));
    AFMM_TRY(dalloc_t(p, &p->t_geo, 2 * nf));
    for (int set = 0; set < 2; ++set) {
        int64_t n = set == 0 ? ns : nf;
        int64_t npad = pow2_at_least(n);
        const double *r = set == 0 ? src_r : tgt_r, *z = set == 0 ? src_z : tgt_z;
        k_keys<<<nblk(npad), 256, 0, st>>>(r, z, n, npad, p->r0, p->z0, s16, srt);
        AFMM_LAUNCH_CHECK();
        AFMM_TRY(bitonic_sort(srt, npad, st));
        if (set == 0)
            k_gather_sorted<<<nblk(n), 256, 0, st>>>(srt, n, r, z, p->s_r, p->s_z, p->s_geo, p->s_perm, p->s_key);
        else
            k_gather_sorted<<<nblk(n), 256, 0, st>>>(srt, n, r, z, p->t_r, p->t_z, p->t_geo, p->t_perm, p->t_key);
        AFMM_LAUNCH_CHECK();
    }
    // ---- depth (uniform tree), or the levels of the adaptive tree
    p->adaptive = p->opt.tree == AFMM_TREE_ADAPTIVE ? 1 : 0;
    if (p->adaptive) AFMM_TRY(build_levels_adaptive(p));
    int d = p->adaptive ? p->d : p->opt.depth_override;
    if (!p->adaptive && d <= 0) {
        unsigned long long *cnt = nullptr;
        AFMM_TRY(dalloc_t(p, &cnt, 17));
        AFMM_CUDA(cudaMemsetAsync(cnt, 0, 17 * sizeof(unsigned long long), st));
        k_depth_counts<<<nblk(ns), 256, 0, st>>>(p->s_key, ns, cnt);
        AFMM_LAUNCH_CHECK();
        unsigned long long hc[17];
        AFMM_TRY(readback(p, hc, cnt, sizeof(hc)));
        d = -1;
        for (int l = 2; l <= 16; ++l)
            if (hc[l] > 0 && (double)ns <= (double)p->opt.leaf_size * (double)hc[l]) {
                d = l;
                break;
            }
        if (d < 0) d = 16;
    }
    if (d < 2 || d > AFMM_MAX_LEVEL) return AFMM_EUNSUPPORTED;
    p->d = d;

    // ---- boxes per level: union of leaf keys, then parents
    if (!p->adaptive) {
        int64_t npad = pow2_at_least(ns + nf);
        k_leaf_union<<<nblk(npad), 256, 0, st>>>(p->s_key, ns, p->t_key, nf, 2 * (16 - d), npad, srt);
        AFMM_LAUNCH_CHECK();
        AFMM_TRY(bitonic_sort(srt, npad, st));
        AFMM_TRY(uniq_keys(p, srt, ns + nf, 0, f, pos, tmp, &p->lv[d].key, &p->lv[d].nbox));
        for (int l = d - 1; l >= 2; --l) {
            int64_t nc = p->lv[l + 1].nbox;
            k_parent_keys<<<nblk(nc), 256, 0, st>>>(p->lv[l + 1].key, nc, srt);
            AFMM_LAUNCH_CHECK();
            AFMM_TRY(uniq_keys(p, srt, nc, 0, f, pos, tmp, &p->lv[l].key, &p->lv[l].nbox));
        }
    }
    // ---- per-level tables
    for (int l = 2; l <= d; ++l) {
        Level &v = p->lv[l];
        int64_t nb = v.nbox;
        if (nb >= (1 << 24)) return AFMM_EUNSUPPORTED;  // S2L unit keys hold 24-bit box indices
        if (!p->adaptive) {  // (the adaptive tree builds these with its levels)
            AFMM_TRY(dalloc_t(p, &v.srng, nb));
            AFMM_TRY(dalloc_t(p, &v.trng, nb));
            k_box_ranges<<<nblk(nb), 256, 0, st>>>(v.key, nb, 2 * (16 - l), p->s_key, ns, p->t_key, nf, v.srng, v.trng);
            AFMM_LAUNCH_CHECK();
            if (l >= 3) {
                AFMM_TRY(dalloc_t(p, &v.parent, nb));
                k_parents<<<nblk(nb), 256, 0, st>>>(v.key, nb, p->lv[l - 1].key, p->lv[l - 1].nbox, v.parent);
                AFMM_LAUNCH_CHECK();
                AFMM_TRY(dalloc_t(p, &p->lv[l - 1].child, p->lv[l - 1].nbox));
                k_child_ranges<<<nblk(nb), 256, 0, st>>>(v.parent, nb, p->lv[l - 1].child);
                AFMM_LAUNCH_CHECK();
            }
        }
        AFMM_TRY(dalloc_t(p, &v.s2l, nb * 27));
        k_s2l_table<<<nblk(nb * 27), 256, 0, st>>>(v.key, nb, l, v.s2l);
        AFMM_LAUNCH_CHECK();
        // stations (occupied columns)
        int ncol = 1 << l;
        int32_t *flag = nullptr;
        AFMM_TRY(dalloc_t(p, &flag, ncol));
        AFMM_TRY(dalloc_t(p, &v.station_of_col, ncol));
        AFMM_CUDA(cudaMemsetAsync(flag, 0, ncol * sizeof(int32_t), st));
        k_station_flags<<<nblk(nb), 256, 0, st>>>(v.key, nb, flag);
        AFMM_LAUNCH_CHECK();
        k_i32_to_i64<<<nblk(ncol), 256, 0, st>>>(flag, ncol, f);
        AFMM_LAUNCH_CHECK();
        AFMM_TRY(scan_excl(f, pos, ncol, tmp, st));
        int64_t nst = 0;
        AFMM_TRY(readback(p, &nst, pos + ncol, sizeof(int64_t)));
        v.nstation = (int)nst;
        AFMM_TRY(dalloc_t(p, &v.col_of_station, nst > 0 ? nst : 1));
        k_station_map<<<nblk(ncol), 256, 0, st>>>(flag, ncol, pos, v.station_of_col, v.col_of_station);
        AFMM_LAUNCH_CHECK();
        // S2L units
        int64_t npad = pow2_at_least(nb);
        k_unit_keys<<<nblk(npad), 256, 0, st>>>(v.key, nb, npad, srt);
        AFMM_LAUNCH_CHECK();
        AFMM_TRY(bitonic_sort(srt, npad, st));
        for (int us = 32; us <= 64; us += 32) {
            if (us == 64 && !s2l_tc_enabled(p)) break;  // units of the tensor-core S2L
            k_unit_flags<<<nblk(nb), 256, 0, st>>>(srt, nb, us, f);
            AFMM_LAUNCH_CHECK();
            AFMM_TRY(scan_excl(f, pos, nb, tmp, st));
            int64_t nu = 0;
            AFMM_TRY(readback(p, &nu, pos + nb, sizeof(int64_t)));
            int32_t **ub = us == 32 ? &v.unit_box : &v.unit64_box, **uc = us == 32 ? &v.unit_col : &v.unit64_col;
            (us == 32 ? v.nunit : v.nunit64) = nu;
            AFMM_TRY(dalloc_t(p, ub, (nu > 0 ? nu : 1) * us));
            AFMM_TRY(dalloc_t(p, uc, nu > 0 ? nu : 1));
            AFMM_CUDA(cudaMemsetAsync(*ub, 0xff, (nu > 0 ? nu : 1) * us * sizeof(int32_t), st));
            k_unit_fill<<<nblk(nb), 256, 0, st>>>(srt, nb, us, pos, *ub, *uc);
            AFMM_LAUNCH_CHECK();
        }
    }
    // ---- leaf neighbours and near-field units for both directions
    if (p->adaptive) {
        AFMM_TRY(build_near_adaptive(p));
        unsigned long long *acc = nullptr;
        AFMM_TRY(dalloc_t(p, &acc, 3));
        AFMM_CUDA(cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), st));
        for (int l = 2; l <= d; ++l) {
            const Level &u = p->lv[l];
            k_s2l_count<<<nblk(u.nbox), 256, 0, st>>>(u.s2l, u.trng, u.srng, u.nbox, acc + 1);
            AFMM_LAUNCH_CHECK();
        }
        unsigned long long h[3];
        AFMM_TRY(readback(p, h, acc, sizeof(h)));
        p->s2l_pairs = (int64_t)h[1];
        p->s2l_point_pairs = (int64_t)h[2];
    } else {
        Level &v = p->lv[d];
        int64_t nb = v.nbox;
        AFMM_TRY(dalloc_t(p, &v.nbr, nb * 9));
        k_nbr_table<<<nblk(nb * 9), 256, 0, st>>>(v.key, nb, d, v.nbr);
        AFMM_LAUNCH_CHECK();
        for (int dir = 0; dir < 2; ++dir) {
            const int2 *rng = dir == 0 ? v.trng : v.srng;
            k_near_counts<<<nblk(nb), 256, 0, st>>>(rng, nb, f);
            AFMM_LAUNCH_CHECK();
            AFMM_TRY(scan_excl(f, pos, nb, tmp, st));
            int64_t nu = 0;
            AFMM_TRY(readback(p, &nu, pos + nb, sizeof(int64_t)));
            p->n_near_unit[dir] = nu;
            AFMM_TRY(dalloc_t(p, &p->near_unit[dir], nu > 0 ? nu : 1));
            k_near_fill<<<nblk(nb), 256, 0, st>>>(rng, nb, d, pos, p->near_unit[dir]);
            AFMM_LAUNCH_CHECK();
        }
        unsigned long long *acc = nullptr;
        AFMM_TRY(dalloc_t(p, &acc, 4));
        AFMM_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long), st));
        k_near_pairs<<<nblk(nb), 256, 0, st>>>(v.trng, v.srng, v.nbr, nb, acc);
        AFMM_LAUNCH_CHECK();
        for (int l = 2; l <= d; ++l) {
            const Level &u = p->lv[l];
            k_s2l_count<<<nblk(u.nbox), 256, 0, st>>>(u.s2l, u.trng, u.srng, u.nbox, acc + 1);
            AFMM_LAUNCH_CHECK();
        }
        unsigned long long h[4];
        AFMM_TRY(readback(p, h, acc, sizeof(h)));
        p->near_pairs = (int64_t)h[0];
        p->s2l_pairs = (int64_t)h[1];
        p->s2l_point_pairs = (int64_t)h[2];
        p->near_max_src = (int64_t)h[3];
    }
    p->n_max = nmax;
    return AFMM_OK;
}

}  // namespace afmm
