// Device code of the swap-potential step: cell-sorted Verlet list build,
// the per-centre S pass, the force pass fused with the integrator, and the
// persistent cooperative kernel that runs many time steps per launch.
//
// Method (Ciarella & Ellenbroek, section "The swap potential"):
//   two-body term  v(r) = 4 eps [(sigma/r)^(2n) - (sigma/r)^n]       (Eq. 2b)
//   normalised     vh(r) = 1 (r <= r_min), -v(r)/eps (r > r_min)       (Eq. pot)
//   three-body     v3_ijk = lambda eps vh_ij vh_ik, centre i           (Eq. 3bp)
// With a = sqrt(lambda eps) and S_i = sum_k a_ik vh_ik over the reactive
// partners of i, the three-body energy of centre i is
//   sum_{j<k} a_ij a_ik vh_ij vh_ik = 1/2 sum_j a_ij vh_ij (S_i - a_ij vh_ij)
// and dU3/dvh_ij = a_ij [(S_i - a_ij vh_ij) + (S_j - a_ij vh_ij)], so the
// triplet sum costs O(neighbours) once S is known for every particle: one
// pass forms S, the next forms every pair force from S_i and S_j.  Beyond
// r_min, vh' = -v'/eps_hat, so the total force of a reactive pair is the
// two-body force times (1 - dU3/dvh_ij / eps_hat).
#pragma once

#include "swp_internal.h"

namespace swp {

// ---------------------------------------------------------------------------
// Small helpers

__device__ __forceinline__ long long gtimer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// IEEE operations with one rounding each and no contraction, for the
// distance decisions that must be reproducible bit for bit.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ int packed_of(float w) { return __float_as_int(w); }
__device__ __forceinline__ int packed_of(double w) { return (int)__double_as_longlong(w); }
__device__ __forceinline__ float pack_w(int v, float) { return __int_as_float(v); }
__device__ __forceinline__ double pack_w(int v, double) { return __longlong_as_double((long long)v); }

__device__ __forceinline__ float fix_to_real(long long q, float) { return __ll2float_rn(q) * 0x1p-48f; }
__device__ __forceinline__ double fix_to_real(long long q, double) { return __ll2double_rn(q) * kInvFix; }
__device__ __forceinline__ long long real_to_fix(float x) { return __float2ll_rn(x * 0x1p48f); }
__device__ __forceinline__ long long real_to_fix(double x) { return __double2ll_rn(x * kFix); }

__device__ __forceinline__ const PairP<float>* uni_params(const RunArgs& a, float) { return a.uf; }
__device__ __forceinline__ const PairP<double>* uni_params(const RunArgs& a, double) { return a.ud; }

// Selects the run constant of the arithmetic precision.
__device__ __forceinline__ float pick(float, float f, double) { return f; }
__device__ __forceinline__ double pick(double, float, double d) { return d; }

template <typename R4>
__device__ __forceinline__ int type_of(const R4& p) { return packed_of(p.w) & ((1 << kTypeBits) - 1); }

// Squared minimum-image distance of j from i, in the decision precision;
// returns dx = x_j - x_i (wrapped) for the force evaluation.
template <typename Real, typename R4>
__device__ __forceinline__ Real dist2(const R4& pi, const R4& pj, const Dev<Real>& d, Real& dx,
                                      Real& dy, Real& dz)
{
    dx = sub_rn(pj.x, pi.x);
    dy = sub_rn(pj.y, pi.y);
    dz = sub_rn(pj.z, pi.z);
    if (dx > d.hL[0]) dx = sub_rn(dx, d.L[0]);
    else if (dx < -d.hL[0]) dx = add_rn(dx, d.L[0]);
    if (dy > d.hL[1]) dy = sub_rn(dy, d.L[1]);
    else if (dy < -d.hL[1]) dy = add_rn(dy, d.L[1]);
    if (dz > d.hL[2]) dz = sub_rn(dz, d.L[2]);
    else if (dz < -d.hL[2]) dz = add_rn(dz, d.L[2]);
    Real s = mul_rn(dx, dx);
    s = add_rn(s, mul_rn(dy, dy));
    s = add_rn(s, mul_rn(dz, dz));
    return s;
}

// The same squared distance for a pair already in the list (|x_j - x_i| wraps
// at most once and the wrapped distance is below the list radius, a third of
// the box): k = rint(dx / L) is then the wrap of the branchy form above and
// dx - k L is the same single rounding, so d2 is bit-identical.
__device__ __forceinline__ float wrap_rint(float dx, float L, float iL) { return fmaf(-L, rintf(dx * iL), dx); }
__device__ __forceinline__ double wrap_rint(double dx, double L, double iL) { return fma(-L, rint(dx * iL), dx); }

template <typename Real, typename R4>
__device__ __forceinline__ Real dist2_listed(const R4& pi, const R4& pj, const Dev<Real>& d, Real& dx,
                                             Real& dy, Real& dz)
{
    dx = wrap_rint(sub_rn(pj.x, pi.x), d.L[0], d.iL[0]);
    dy = wrap_rint(sub_rn(pj.y, pi.y), d.L[1], d.iL[1]);
    dz = wrap_rint(sub_rn(pj.z, pi.z), d.L[2], d.iL[2]);
    Real s = mul_rn(dx, dx);
    s = add_rn(s, mul_rn(dy, dy));
    s = add_rn(s, mul_rn(dz, dz));
    return s;
}

template <typename Real>
__device__ __forceinline__ Real ipow(Real b, int e)
{
    // the common exponents n = 10 and n = 6 (e = n/2) by their short chains;
    // e is uniform over a warp, so the branch costs no divergence
    if (e == 5) {
        Real b2 = b * b;
        return b2 * b2 * b;
    }
    if (e == 3) return b * b * b;
    Real r = Real(1);
    while (e) {
        if (e & 1) r *= b;
        e >>= 1;
        if (e) b *= b;
    }
    return r;
}

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Eq. 2b at squared distance r2: v and f = -(dv/dr)/r.
template <typename Real>
__device__ __forceinline__ void lj_eval(const PairP<Real>& p, Real r2, Real& v, Real& f)
{
    Real ir2 = recip(r2);
    Real s2 = p.sig2 * ir2;
    Real x = ipow(s2, p.nhalf);
    if (p.odd) x *= sqrt(s2);
    Real x2 = x * x;
    v = p.four_eps * (x2 - x);
    f = p.four_eps * p.n_real * (Real(2) * x2 - x) * ir2;
}

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Three standard normals for (seed, step, tag): counter (tag, step lo,
// step hi, 1), key (seed lo, seed hi), Box-Muller on (u0,u1) and (u2,u3).
__device__ __forceinline__ void normals3(unsigned long long seed, long long step, unsigned tag,
                                         float z[3])
{
    uint4 w = philox4x32_10(make_uint4(tag, (unsigned)step, (unsigned)((unsigned long long)step >> 32), 1u),
                            make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const float s32 = 2.3283064365386963e-10f;
    float u0 = (__uint2float_rn(w.x) + 0.5f) * s32;
    float u1 = (__uint2float_rn(w.y) + 0.5f) * s32;
    float u2 = (__uint2float_rn(w.z) + 0.5f) * s32;
    float u3 = (__uint2float_rn(w.w) + 0.5f) * s32;
    float ra = sqrtf(-2.0f * logf(u0));
    float rb = sqrtf(-2.0f * logf(u2));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    z[0] = ra * cs;
    z[1] = ra * sn;
    z[2] = rb * cospif(2.0f * u3);
}

__device__ __forceinline__ void normals3(unsigned long long seed, long long step, unsigned tag,
                                         double z[3])
{
    uint4 w = philox4x32_10(make_uint4(tag, (unsigned)step, (unsigned)((unsigned long long)step >> 32), 1u),
                            make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const double s32 = 2.3283064365386962890625e-10;
    double u0 = ((double)w.x + 0.5) * s32;
    double u1 = ((double)w.y + 0.5) * s32;
    double u2 = ((double)w.z + 0.5) * s32;
    double u3 = ((double)w.w + 0.5) * s32;
    double ra = sqrt(-2.0 * log(u0));
    double rb = sqrt(-2.0 * log(u2));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    z[0] = ra * cs;
    z[1] = ra * sn;
    z[2] = rb * cospi(2.0 * u3);
}

template <int LANES>
__device__ __forceinline__ unsigned group_mask()
{
    if (LANES == 32) return 0xffffffffu;
    unsigned lw = threadIdx.x & 31;
    return ((1u << (LANES & 31)) - 1u) << (lw & ~(unsigned)(LANES - 1));
}

template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, LANES);
    return v;
}

// ---------------------------------------------------------------------------
// Grid barrier for the cooperative launch: split arrive / wait, every wait
// bounded in time; on expiry the status word gets kStatusTimeout and every
// block leaves the kernel.

struct BarState {
    unsigned long long target;  // valid in thread 0
};

__device__ __forceinline__ void bar_arrive(Ctl* ctl, BarState& b)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long old = atomicAdd(&ctl->barrier, 1ull);
        b.target = (old / gridDim.x + 1ull) * gridDim.x;
    }
}

__device__ __forceinline__ bool bar_wait(Ctl* ctl, const BarState& b, long long timeout_ns,
                                         int where, int* s_ok)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        int spins = 0;
        long long t0 = 0;
        while (ld_acquire(&ctl->barrier) < b.target) {
            if (++spins < 64) continue;
            if (spins == 64) t0 = gtimer_ns();
            if (ld_relaxed(&ctl->status) & kStatusTimeout) {
                ok = 0;
                break;
            }
            if (gtimer_ns() - t0 > timeout_ns) {
                atomicOr(&ctl->status, kStatusTimeout);
                ctl->timeout_at = where;
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Block reductions

// Sums the per-thread accumulators over the block into partials[slot][q]:
// warp shuffles, then one warp combines the warp sums, in the arithmetic
// precision (at most 1024 terms per block); the block totals are summed over
// blocks in FP64 (reduce_thermo).  FP64 runs at a small fraction of the FP32
// rate on this part, so it is kept out of the per-thread work.
template <typename Real>
__device__ __forceinline__ void block_thermo(const Real* acc, double* out, double* shd)
{
    Real* sh = (Real*)shd;  // kNQA * 32 values
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < kNQA; q++) {
        Real v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[q * 32 + warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
        for (int q = 0; q < kNQA; q++) {
            Real v = lane < nw ? sh[q * 32 + lane] : Real(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) out[q] = (double)v;
        }
        if (lane < kNQ - kNQA) out[kNQA + lane] = 0.0;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(float v, float* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float m = 0.0f;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; w++) m = fmaxf(m, sh[w]);
    __syncthreads();
    return m;  // valid in thread 0
}

__device__ __forceinline__ int block_max_int(int v, int* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int m = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; w++) m = max(m, sh[w]);
    __syncthreads();
    return m;  // valid in thread 0
}

// Exclusive scan of one int per thread over the block (block 0 only).
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < nw) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    int base = warp > 0 ? sh[warp - 1] : 0;
    *total = sh[nw - 1];
    __syncthreads();
    return base + x - v;
}

// ---------------------------------------------------------------------------
// Neighbour-list rebuild phases (K-a): bin by cell, counting sort with a
// deterministic order inside each cell, gather every per-particle array into
// the sorted order, then one row per particle from the 27-cell stencil.

template <typename Real>
__device__ __forceinline__ void cell_coords(const Dev<Real>& d, const typename Dev<Real>::R4& p,
                                            int& cx, int& cy, int& cz)
{
    cx = (int)(p.x * d.inv_cw[0]);
    cy = (int)(p.y * d.inv_cw[1]);
    cz = (int)(p.z * d.inv_cw[2]);
    cx = min(max(cx, 0), d.nc[0] - 1);
    cy = min(max(cy, 0), d.nc[1] - 1);
    cz = min(max(cz, 0), d.nc[2] - 1);
}

template <typename Real>
__device__ void ph_bin(const Dev<Real>& d, int pc, int t, int nt)
{
    for (int p = t; p < d.n; p += nt) {
        int cx, cy, cz;
        cell_coords(d, d.pos[pc][p], cx, cy, cz);
        int r = __ldg(&d.cell_rank[(cz * d.nc[1] + cy) * d.nc[0] + cx]);
        d.perm[p] = r;  // temporarily: cell rank of old slot p
        atomicAdd(&d.cell_cnt[r], 1);
    }
}

// Parallel exclusive scan of the cell counts in two steps.  Block b owns the
// contiguous chunk [b*ch, (b+1)*ch) of cells.  Step 1: each block sums its
// chunk into bsum[b].  Step 2 (after a grid barrier): each block adds up the
// sums of the blocks before it, scans its own chunk, writes cell_start and
// cell_fill, and zeroes the counts it consumed (so the next build starts
// from zero without a separate pass).
__device__ __forceinline__ int block_sum_int(int v, int* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; w++) t += sh[w];
    __syncthreads();
    return t;
}

template <typename Real>
__device__ void ph_chunk_sums(const Dev<Real>& d, int* sh)
{
    const int ch = (d.ncell + gridDim.x - 1) / gridDim.x;
    const int beg = min((int)blockIdx.x * ch, d.ncell), end = min(beg + ch, d.ncell);
    int v = 0;
    for (int c = beg + threadIdx.x; c < end; c += blockDim.x) v += d.cell_cnt[c];
    int t = block_sum_int(v, sh);
    if (threadIdx.x == 0) d.bsum[blockIdx.x] = t;
}

template <typename Real>
__device__ void ph_chunk_scan(const Dev<Real>& d, int* sh)
{
    const int ch = (d.ncell + gridDim.x - 1) / gridDim.x;
    const int beg = min((int)blockIdx.x * ch, d.ncell), end = min(beg + ch, d.ncell);
    int v = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) v += d.bsum[b];
    int base = block_sum_int(v, sh);
    // scan the chunk in pieces of blockDim.x cells
    for (int c0 = beg; c0 < end; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int cnt = c < end ? d.cell_cnt[c] : 0;
        int total;
        int ex = block_excl_scan(cnt, sh, &total);
        if (c < end) {
            d.cell_start[c] = base + ex;
            d.cell_fill[c] = base + ex;
            d.cell_cnt[c] = 0;
        }
        base += total;
    }
    if (end == d.ncell && beg < end && threadIdx.x == 0) d.cell_start[d.ncell] = base;
}

template <typename Real>
__device__ void ph_scatter(const Dev<Real>& d, int t, int nt)
{
    // perm[p] holds the rank of p's cell; write the slot order into cell_of
    // (reused as the inverse map's scratch) then back into perm.
    for (int p = t; p < d.n; p += nt) {
        int r = d.perm[p];
        int q = atomicAdd(&d.cell_fill[r], 1);
        d.cell_fill[d.ncell + q] = p;  // scratch area after the fill counters
    }
}

// Sorts each cell's members by old slot (deterministic order), into perm.
template <typename Real>
__device__ void ph_cell_sort(const Dev<Real>& d, int t, int nt)
{
    const int* src = d.cell_fill + d.ncell;
    for (int c = t; c < d.ncell; c += nt) {
        int s = d.cell_start[c], e = d.cell_start[c + 1];
        for (int a = s; a < e; a++) d.perm[a] = src[a];
        for (int a = s + 1; a < e; a++) {
            int v = d.perm[a], b = a - 1;
            while (b >= s && d.perm[b] > v) {
                d.perm[b + 1] = d.perm[b];
                b--;
            }
            d.perm[b + 1] = v;
        }
    }
}

template <typename Real>
__device__ void ph_gather(const Dev<Real>& d, int pc, int ac, int t, int nt)
{
    const int n = d.n;
    for (int q = t; q < n; q += nt) {
        int p = d.perm[q];
        d.pos[pc ^ 1][q] = d.pos[pc][p];
        d.vel[ac ^ 1][q] = d.vel[ac][p];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            d.xq[ac ^ 1][c * n + q] = d.xq[ac][c * n + p];
            d.img[ac ^ 1][c * n + q] = d.img[ac][c * n + p];
        }
    }
}

// ---------------------------------------------------------------------------
// Block ownership and the compact neighbour list.
//
// Block b of a G-block launch owns the contiguous (Morton-ordered, hence
// spatially compact) particle range [b*Pb, min((b+1)*Pb, n)), Pb = ceil(n/G),
// processed in sub-chunks of at most blockDim.x particles.  The neighbour
// entries of a sub-chunk are stored contiguously in the block's region of the
// list buffer (capacity Pb * max_nn entries): first the reactive entries of
// all its particles (in particle order), then the other entries.  Entry e
// holds the partner slot ent_j[e] and the owner's index inside its sub-chunk
// ent_o[e]; pinfo[p] = (first reactive entry, n_reactive, first other entry,
// n_other).  The S and F passes then give one thread to one entry, so the
// lanes of a warp neither idle on short rows nor diverge between the two
// kinds of pair, and each owner thread sums its entries in entry order.

template <typename Real>
__device__ __forceinline__ void block_range(const Dev<Real>& d, int& b0, int& b1)
{
    const int Pb = (d.n + (int)gridDim.x - 1) / (int)gridDim.x;
    b0 = min((int)blockIdx.x * Pb, d.n);
    b1 = min(b0 + Pb, d.n);
}

template <int LB>
__device__ __forceinline__ int group_excl_scan(int v, unsigned mask, int lane, int* total)
{
    int x = v;
#pragma unroll
    for (int o = 1; o < LB; o <<= 1) {
        int y = __shfl_up_sync(mask, x, o, LB);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(mask, x, LB - 1, LB);
    return x - v;
}

// The 27 stencil cells of a particle, split over the LB lanes of its group:
// lane l takes cells l, l+LB, ...; their [start, end) slot ranges.
template <typename Real, int LB>
struct Stencil {
    static constexpr int NU = (27 + LB - 1) / LB;
    int cs[NU], ce[NU];

    __device__ __forceinline__ void load(const Dev<Real>& d, const typename Dev<Real>::R4& pi, int lane)
    {
        int cx, cy, cz;
        cell_coords(d, pi, cx, cy, cz);
#pragma unroll
        for (int u = 0; u < NU; u++) {
            const int c = lane + LB * u;
            cs[u] = ce[u] = 0;
            if (c < 27) {
                int x = cx + c % 3 - 1, y = cy + (c / 3) % 3 - 1, z = cz + c / 9 - 1;
                x = x < 0 ? x + d.nc[0] : (x >= d.nc[0] ? x - d.nc[0] : x);
                y = y < 0 ? y + d.nc[1] : (y >= d.nc[1] ? y - d.nc[1] : y);
                z = z < 0 ? z + d.nc[2] : (z >= d.nc[2] ? z - d.nc[2] : z);
                const int r = __ldg(&d.cell_rank[(z * d.nc[1] + y) * d.nc[0] + x]);
                cs[u] = d.cell_start[r];
                ce[u] = d.cell_start[r + 1];
            }
        }
    }
};

// Visits every listed partner of slot i among this lane's stencil cells:
// fn(q, reactive).  The decision is the exact squared distance against the
// pair's list radius.
template <typename Real, int LB, typename Fn>
__device__ __forceinline__ void for_partners(const Dev<Real>& d, const PairP<Real>* tab,
                                             const typename Dev<Real>::R4* pos,
                                             const Stencil<Real, LB>& st, int i,
                                             const typename Dev<Real>::R4& pi, Fn fn)
{
    typedef typename Dev<Real>::R4 R4;
    const int ti = type_of(pi);
#pragma unroll
    for (int u = 0; u < Stencil<Real, LB>::NU; u++)
        for (int q = st.cs[u]; q < st.ce[u]; q++) {
            if (q == i) continue;
            const R4 pj = pos[q];
            const PairP<Real>& p = tab[ti * d.ntypes + type_of(pj)];
            Real dx, dy, dz;
            if (dist2(pi, pj, d, dx, dy, dz) < p.rlist2) fn(q, p.kind == KIND_SWAP);
        }
}

// Builds the block's entries (K-a, last step).  cnt: blockDim.x int2 of
// shared memory.  Returns the block's total entry count divided by its
// particle count (rounded up), the row length a capacity check needs.
template <typename Real, int LB>
__device__ int ph_build_block(const Dev<Real>& d, const PairP<Real>* tab, int pc, int2* cnt,
                              int* sh, int* overflow)
{
    typedef typename Dev<Real>::R4 R4;
    const R4* pos = d.pos[pc];
    const int lane = threadIdx.x % LB, grp = threadIdx.x / LB, ngrp = blockDim.x / LB;
    const unsigned mask = group_mask<LB>();
    int b0, b1;
    block_range(d, b0, b1);
    const int Pb = (d.n + (int)gridDim.x - 1) / (int)gridDim.x;
    const long long cap_beg = (long long)blockIdx.x * Pb * d.max_nn;
    const long long cap_end = cap_beg + (long long)Pb * d.max_nn;
    long long base = cap_beg;
    for (int q0 = b0; q0 < b1; q0 += blockDim.x) {
        const int P = min((int)blockDim.x, b1 - q0);
        // 1. partner counts per particle
        for (int t = grp; t < P; t += ngrp) {
            const int i = q0 + t;
            const R4 pi = pos[i];
            Stencil<Real, LB> st;
            st.load(d, pi, lane);
            int cr = 0, cw = 0;
            for_partners<Real, LB>(d, tab, pos, st, i, pi, [&](int, bool r) { r ? cr++ : cw++; });
#pragma unroll
            for (int o = LB / 2; o > 0; o >>= 1) {
                cr += __shfl_xor_sync(mask, cr, o, LB);
                cw += __shfl_xor_sync(mask, cw, o, LB);
            }
            if (lane == 0) cnt[t] = make_int2(cr, cw);
        }
        __syncthreads();
        // 2. entry offsets: reactive block, then the others
        const int t = threadIdx.x;
        const int2 c = t < P ? cnt[t] : make_int2(0, 0);
        int Er, Ew;
        const int offr = block_excl_scan(c.x, sh, &Er);
        const int offw = block_excl_scan(c.y, sh, &Ew);
        const bool fits = base + Er + Ew <= cap_end;
        if (t < P)
            d.pinfo[q0 + t] = make_int4((int)(base + offr), c.x, (int)(base + Er + offw), c.y);
        if (!fits && t == 0) *overflow = 1;
        __syncthreads();
        // 3. entries (lane order inside each particle's run)
        if (fits)
            for (int tt = grp; tt < P; tt += ngrp) {
                const int i = q0 + tt;
                const R4 pi = pos[i];
                const int4 inf = d.pinfo[i];
                Stencil<Real, LB> st;
                st.load(d, pi, lane);
                int cr = 0, cw = 0;
                for_partners<Real, LB>(d, tab, pos, st, i, pi, [&](int, bool r) { r ? cr++ : cw++; });
                int tr, tw;
                int er = inf.x + group_excl_scan<LB>(cr, mask, lane, &tr);
                int ew = inf.z + group_excl_scan<LB>(cw, mask, lane, &tw);
                for_partners<Real, LB>(d, tab, pos, st, i, pi, [&](int q, bool r) {
                    const int e = r ? er++ : ew++;
                    d.ent_j[e] = q;
                    d.ent_o[e] = (unsigned short)tt;
                });
            }
        base += Er + Ew;
        __syncthreads();
    }
    const int np = b1 - b0;
    return np > 0 ? (int)((base - cap_beg + np - 1) / np) : 0;
}

// ---------------------------------------------------------------------------
// UNI: every reactive type pair has the same coefficients (ps) and so has
// every other interacting pair (pw); they are then read from the
// kernel-parameter constant bank instead of the shared-memory table, which
// costs neither a lookup nor registers.
template <typename Real, bool UNI>
__device__ __forceinline__ const PairP<Real>& pair_of(const PairP<Real>* tab, int ti, int tj, int nt,
                                                    const PairP<Real>& uni)
{
    return UNI ? uni : tab[ti * nt + tj];
}

// Shared-memory staging of one sub-chunk (dynamic shared memory).
template <typename Real>
struct Stage {
    typedef typename Dev<Real>::R4 R4;
    R4* pos;        // [blockDim.x] positions of the sub-chunk's particles
    R4* vel;        // [blockDim.x] their velocities (asynchronous copy)
    long long* xq;  // [3 * blockDim.x] their fixed-point positions (asynchronous copy)
    int4* info;     // [blockDim.x] their pinfo
    Real* S;        // [blockDim.x] their S
    Real* w;        // [3 * wave] per-entry results of one wave
    int wave;       // entries per wave

    static constexpr int kWave = sizeof(Real) == 4 ? 8192 : 3072;
    static size_t bytes(int block)
    {
        return (size_t)block * (2 * sizeof(R4) + 3 * sizeof(long long) + sizeof(int4) + sizeof(Real)) +
               (size_t)3 * kWave * sizeof(Real);
    }
    __device__ void carve(unsigned char* base)
    {
        const size_t B = blockDim.x;
        pos = (R4*)base;
        vel = (R4*)(base + B * sizeof(R4));
        xq = (long long*)(base + 2 * B * sizeof(R4));
        info = (int4*)(base + B * (2 * sizeof(R4) + 3 * sizeof(long long)));
        S = (Real*)(base + B * (2 * sizeof(R4) + 3 * sizeof(long long) + sizeof(int4)));
        w = (Real*)(base + B * (2 * sizeof(R4) + 3 * sizeof(long long) + sizeof(int4) + sizeof(Real)));
        wave = kWave;
    }
};

// Asynchronous global -> shared copies (no register staging).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename R4>
__device__ __forceinline__ void cp_async_r4(R4* smem, const R4* gmem)
{
    if (sizeof(R4) == 16) {
        cp_async(smem, gmem, 16);
    } else {
        cp_async(smem, gmem, 16);
        cp_async((char*)smem + 16, (const char*)gmem + 16, 16);
    }
}

// ---------------------------------------------------------------------------
// S pass (K-b1): S_i = sum over reactive partners k inside r_cut of a vh(r_ik).

template <typename Real, bool UNI>
__device__ void s_pass_block(const Dev<Real>& d, const PairP<Real>* tab, int pc, Stage<Real>& sm,
                             const PairP<Real>& ps)
{
    typedef typename Dev<Real>::R4 R4;
    const R4* pos = d.pos[pc];
    int b0, b1;
    block_range(d, b0, b1);
    const int t = threadIdx.x;
    for (int q0 = b0; q0 < b1; q0 += blockDim.x) {
        const int P = min((int)blockDim.x, b1 - q0);
        if (t < P) {
            sm.pos[t] = pos[q0 + t];
            sm.info[t] = d.pinfo[q0 + t];
        }
        __syncthreads();
        const int e_beg = sm.info[0].x;
        const int e_end = sm.info[P - 1].x + sm.info[P - 1].y;
        Real s = Real(0);
        for (int wb = e_beg; wb < e_end; wb += sm.wave) {
            const int we = min(wb + sm.wave, e_end);
            for (int e = wb + t; e < we; e += blockDim.x) {
                const int j = d.ent_j[e];
                const int o = d.ent_o[e];
                const R4 pj = pos[j];
                const R4 pi = sm.pos[o];
                const PairP<Real>& p = pair_of<Real, UNI>(tab, type_of(pi), type_of(pj), d.ntypes, ps);
                Real dx, dy, dz;
                const Real r2 = dist2_listed(pi, pj, d, dx, dy, dz);
                Real sv = Real(0);
                if (r2 < p.rc2) {
                    Real vh = Real(1);
                    if (r2 > p.rmin2) {
                        Real v, f;
                        lj_eval(p, r2, v, f);
                        vh = (p.vshift - v) * p.inv_epshat;
                    }
                    sv = p.a * vh;
                }
                sm.w[e - wb] = sv;
            }
            __syncthreads();
            if (t < P) {
                const int4 inf = sm.info[t];
                const int k0 = max(inf.x, wb), k1 = min(inf.x + inf.y, we);
                for (int k = k0; k < k1; k++) s += sm.w[k - wb];
            }
            __syncthreads();
        }
        if (t < P) d.S[q0 + t] = s;
    }
}

// ---------------------------------------------------------------------------
// Force pass (K-b2) fused with the integrator (K-c).
//
// flags: closing = finish the current step with the second half kick;
//        opening = start the next step: half kick, half drift, (Langevin O),
//                  half drift, write the new snapshot into pos[pc^1];
//        store   = keep the forces (for a later opening or a read-out).
enum { F_CLOSING = 1, F_OPENING = 2, F_STORE = 4 };

template <typename Real>
struct Acc {
    Real q[kNQA];
};

// Per-particle integrator inputs, loaded before the force gathers so that
// their latency overlaps the entry work.
template <typename Real>
struct PState {
    typename Dev<Real>::R4 v;
    long long q[3];
};

template <typename Real>
__device__ __forceinline__ void load_pstate(const Dev<Real>& d, int ac, int i, int flags,
                                            PState<Real>& ps)
{
    const int n = d.n;
    ps.v = d.vel[ac][i];
    if (flags & F_OPENING) {
#pragma unroll
        for (int c = 0; c < 3; c++) ps.q[c] = d.xq[ac][c * n + i];
    }
}

// Adds a displacement to one fixed-point coordinate, wraps it into the box
// (counting the image) and returns the new snapshot coordinate.
template <typename Real>
__device__ __forceinline__ Real advance_fix(const Dev<Real>& d, int ac, int i, int c, long long q0,
                                            Real dx)
{
    const int n = d.n;
    long long q = q0 + real_to_fix(dx);
    const long long Lq = d.Lq[c];
    if (q >= Lq) {
        q -= Lq;
        d.img[ac][c * n + i] += 1;
    } else if (q < 0) {
        q += Lq;
        d.img[ac][c * n + i] -= 1;
    }
    d.xq[ac][c * n + i] = q;
    return fix_to_real(q, Real(0));
}

// Advances particle i given its force.  Returns the squared displacement of
// this step's drift (0 when not opening).
template <typename Real>
__device__ __forceinline__ float integrate_one(const Dev<Real>& d, const RunArgs& a, int pc,
                                               int ac, int i, Real fx, Real fy, Real fz,
                                               int flags, long long step, PState<Real>& st,
                                               Real wbits, Acc<Real>& acc)
{
    typedef typename Dev<Real>::R4 R4;
    R4 v = st.v;
    const Real im = v.w;
    const Real hdt = pick(Real(0), a.hdt_f, a.hdt_d);
    if (flags & F_CLOSING) {
        v.x += hdt * fx * im;
        v.y += hdt * fy * im;
        v.z += hdt * fz * im;
    }
    acc.q[Q_K] += Real(0.5) * (v.x * v.x + v.y * v.y + v.z * v.z) / im;
    float disp2 = 0.0f;
    if (flags & F_OPENING) {
        v.x += hdt * fx * im;
        v.y += hdt * fy * im;
        v.z += hdt * fz * im;
        Real ddx = hdt * v.x, ddy = hdt * v.y, ddz = hdt * v.z;
        if (a.langevin) {
            Real z[3];
            normals3(a.seed, step, (unsigned)(packed_of(wbits) >> kTypeBits), z);
            const Real c1 = pick(Real(0), a.c1_f, a.c1_d);
            const Real sd = pick(Real(0), a.c2_f, a.c2_d) * sqrt(im);
            v.x = c1 * v.x + sd * z[0];
            v.y = c1 * v.y + sd * z[1];
            v.z = c1 * v.z + sd * z[2];
        }
        ddx += hdt * v.x;
        ddy += hdt * v.y;
        ddz += hdt * v.z;
        disp2 = (float)(ddx * ddx + ddy * ddy + ddz * ddz);
        R4 np;
        np.x = advance_fix(d, ac, i, 0, st.q[0], ddx);
        np.y = advance_fix(d, ac, i, 1, st.q[1], ddy);
        np.z = advance_fix(d, ac, i, 2, st.q[2], ddz);
        np.w = wbits;
        d.pos[pc ^ 1][i] = np;
    }
    d.vel[ac][i] = v;
    return disp2;
}

// One entry's pair force on its owner (returned as the components of
// f (x_i - x_j)), with the entry's share of energies, virial and bond count.
// REACT: a reactive pair (two-body plus the three-body factor); else a
// purely two-body pair.
template <typename Real, bool UNI, bool REACT>
__device__ __forceinline__ void entry_force(const Dev<Real>& d, const PairP<Real>* tab,
                                            const typename Dev<Real>::R4& pi,
                                            const typename Dev<Real>::R4& pj, Real Si, Real Sj,
                                            const PairP<Real>& pu, Acc<Real>& acc, Real& fx,
                                            Real& fy, Real& fz)
{
    Real dx, dy, dz;
    const Real r2 = dist2_listed(pi, pj, d, dx, dy, dz);
    fx = fy = fz = Real(0);
    const PairP<Real>& p = pair_of<Real, UNI>(tab, type_of(pi), type_of(pj), d.ntypes, pu);
    if (!(r2 < p.rc2)) return;
    Real v, ft;
    lj_eval(p, r2, v, ft);
    acc.q[Q_U2] += Real(0.5) * (v + p.ushift);
    if (REACT) {
        Real vh = Real(1);
        if (r2 > p.rmin2) {
            vh = (p.vshift - v) * p.inv_epshat;
            const Real h = p.a * (Si + Sj - Real(2) * p.a * vh);
            ft *= Real(1) - h * p.inv_epshat;
        }
        acc.q[Q_U3] += Real(0.5) * p.a * vh * (Si - p.a * vh);
        if (r2 < p.rbond2) acc.q[Q_BONDS] += Real(0.5);
    }
    fx = -ft * dx;
    fy = -ft * dy;
    fz = -ft * dz;
    const Real hf = Real(0.5) * ft;
    acc.q[Q_W0 + 0] += hf * dx * dx;
    acc.q[Q_W0 + 1] += hf * dy * dy;
    acc.q[Q_W0 + 2] += hf * dz * dz;
    acc.q[Q_W0 + 3] += hf * dx * dy;
    acc.q[Q_W0 + 4] += hf * dx * dz;
    acc.q[Q_W0 + 5] += hf * dy * dz;
}

template <typename Real, bool UNI>
__device__ float f_pass_block(const Dev<Real>& d, const PairP<Real>* tab, const RunArgs& a, int pc,
                              int ac, int flags, long long step, Stage<Real>& sm, Acc<Real>& acc,
                              const PairP<Real>& ps, const PairP<Real>& pw)
{
    typedef typename Dev<Real>::R4 R4;
    const R4* pos = d.pos[pc];
    int b0, b1;
    block_range(d, b0, b1);
    const int t = threadIdx.x;
    const int n = d.n;
    float dmax = 0.0f;
    for (int q0 = b0; q0 < b1; q0 += blockDim.x) {
        const int P = min((int)blockDim.x, b1 - q0);
        if (t < P) {
            const int i = q0 + t;
            // integrator inputs: asynchronous copies, waited for after the entries
            cp_async_r4(&sm.vel[t], &d.vel[ac][i]);
            if (flags & F_OPENING)
                for (int c = 0; c < 3; c++) cp_async(&sm.xq[3 * t + c], &d.xq[ac][c * n + i], 8);
            cp_async_commit();
            sm.pos[t] = pos[i];
            sm.S[t] = d.S[i];
            sm.info[t] = d.pinfo[i];
        }
        __syncthreads();
        const int e_beg = sm.info[0].x;
        const int e_rend = sm.info[P - 1].x + sm.info[P - 1].y;
        const int e_end = sm.info[P - 1].z + sm.info[P - 1].w;
        Real fx = 0, fy = 0, fz = 0;
        for (int wb = e_beg; wb < e_end; wb += sm.wave) {
            const int we = min(wb + sm.wave, e_end);
            for (int e = wb + t; e < we; e += blockDim.x) {
                const int j = d.ent_j[e];
                const int o = d.ent_o[e];
                const R4 pj = pos[j];
                Real ex, ey, ez;
                if (e < e_rend)
                    entry_force<Real, UNI, true>(d, tab, sm.pos[o], pj, sm.S[o], d.S[j], ps, acc, ex, ey, ez);
                else
                    entry_force<Real, UNI, false>(d, tab, sm.pos[o], pj, Real(0), Real(0), pw, acc, ex, ey, ez);
                sm.w[3 * (e - wb) + 0] = ex;
                sm.w[3 * (e - wb) + 1] = ey;
                sm.w[3 * (e - wb) + 2] = ez;
            }
            __syncthreads();
            if (t < P) {
                const int4 inf = sm.info[t];
                int k0 = max(inf.x, wb), k1 = min(inf.x + inf.y, we);
                for (int k = k0; k < k1; k++) {
                    fx += sm.w[3 * (k - wb) + 0];
                    fy += sm.w[3 * (k - wb) + 1];
                    fz += sm.w[3 * (k - wb) + 2];
                }
                k0 = max(inf.z, wb);
                k1 = min(inf.z + inf.w, we);
                for (int k = k0; k < k1; k++) {
                    fx += sm.w[3 * (k - wb) + 0];
                    fy += sm.w[3 * (k - wb) + 1];
                    fz += sm.w[3 * (k - wb) + 2];
                }
            }
            __syncthreads();
        }
        if (t < P) {
            const int i = q0 + t;
            if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(&d.ctl->status, kStatusNonfinite);
            if (flags & F_STORE) {
                R4 f;
                f.x = fx;
                f.y = fy;
                f.z = fz;
                f.w = Real(0);
                d.force[i] = f;
            }
            cp_async_wait_all();
            PState<Real> st;
            st.v = sm.vel[t];
            if (flags & F_OPENING)
                for (int c = 0; c < 3; c++) st.q[c] = sm.xq[3 * t + c];
            dmax = fmaxf(dmax, integrate_one(d, a, pc, ac, i, fx, fy, fz, flags, step, st, sm.pos[t].w, acc));
        }
        __syncthreads();
    }
    return dmax;
}

// Opening half of a step from stored forces (start of a run).
template <typename Real>
__device__ __forceinline__ float open_from_stored(const Dev<Real>& d, const RunArgs& a, int pc,
                                                  int ac, int i, long long step)
{
    typedef typename Dev<Real>::R4 R4;
    const R4 f = d.force[i];
    const R4 pi = d.pos[pc][i];
    PState<Real> st;
    load_pstate(d, ac, i, F_OPENING, st);
    Acc<Real> unused;
#pragma unroll
    for (int q = 0; q < kNQA; q++) unused.q[q] = Real(0);
    return integrate_one(d, a, pc, ac, i, f.x, f.y, f.z, F_OPENING, step, st, pi.w, unused);
}

// ---------------------------------------------------------------------------
// The persistent step kernel.  One cooperative launch advances a.nsteps time
// steps (or only rebuilds, or only brings the forces up to date), with two
// grid barriers per step and a rebuild whenever the accumulated displacement
// bound can let an unlisted pair come inside its cut-off.

template <typename Real, int LB, bool UNI>
struct Runner {
    typedef typename Dev<Real>::R4 R4;
    const Dev<Real>& d;
    const RunArgs& a;
    PairP<Real>* tab;
    double* sh_red;
    int* sh_int;
    float* sh_f;
    int* s_ok;
    float* s_disp;
    int2* sh_cnt;
    Stage<Real> sm;
    Ctl* ctl;
    int gt, gn;
    int pc, ac;
    long long rebuilds;
    BarState bs;
    const PairP<Real>& ps;  // uniform coefficients (UNI), in the kernel-parameter bank
    const PairP<Real>& pw;

    __device__ Runner(const Dev<Real>& d_, const RunArgs& a_, PairP<Real>* tab_, double* sr,
                      int* si, float* sf, int* so, float* sd, unsigned char* dyn)
        : d(d_), a(a_), tab(tab_), sh_red(sr), sh_int(si), sh_f(sf), s_ok(so), s_disp(sd),
          ctl(d_.ctl), ps(uni_params(a_, Real(0))[0]), pw(uni_params(a_, Real(0))[1])
    {
        gt = blockIdx.x * blockDim.x + threadIdx.x;
        gn = gridDim.x * blockDim.x;
        rebuilds = 0;
        bs.target = 0;
        sm.carve(dyn);
        sh_cnt = (int2*)sm.w;  // the build's counts reuse the wave buffer
    }

    __device__ __forceinline__ bool barrier(int where)
    {
        bar_arrive(ctl, bs);
        return bar_wait(ctl, bs, a.timeout_ns, where, s_ok);
    }

    // 0: ok; 1: the list overflowed its capacity; 2: a wait timed out.
    __device__ int rebuild()
    {
        if (threadIdx.x == 0 && blockIdx.x == 0) {
            ctl->max_row = 0;
            ctl->overflow = 0;
        }
        ph_bin(d, pc, gt, gn);  // cell counts start at zero (see ph_chunk_scan)
        if (!barrier(1)) return 2;
        ph_chunk_sums(d, sh_int);
        if (!barrier(2)) return 2;
        ph_chunk_scan(d, sh_int);
        if (!barrier(3)) return 2;
        ph_scatter(d, gt, gn);
        if (!barrier(4)) return 2;
        ph_cell_sort(d, gt, gn);
        if (!barrier(5)) return 2;
        ph_gather(d, pc, ac, gt, gn);
        pc ^= 1;
        ac ^= 1;
        if (!barrier(6)) return 2;
        int ovf = 0;
        const int need = ph_build_block<Real, LB>(d, tab, pc, sh_cnt, sh_int, &ovf);
        if (threadIdx.x == 0) {
            atomicMax(&ctl->max_row, need);
            if (ovf) atomicOr(&ctl->overflow, 1);
        }
        if (!barrier(7)) return 2;
        const int any_ovf = ld_relaxed(&ctl->overflow);
        rebuilds++;
        if (threadIdx.x == 0) *s_disp = 0.0f;
        __syncthreads();
        if (any_ovf) {
            if (gt == 0) atomicOr(&ctl->status, kStatusOverflow);
            return 1;
        }
        return 0;
    }

    __device__ void s_pass() { s_pass_block<Real, UNI>(d, tab, pc, sm, ps); }

    __device__ void f_pass(int flags, long long stp, int par)
    {
        Acc<Real> acc;
#pragma unroll
        for (int q = 0; q < kNQA; q++) acc.q[q] = Real(0);
        float dmax = f_pass_block<Real, UNI>(d, tab, a, pc, ac, flags, stp, sm, acc, ps, pw);
        block_thermo(acc.q, d.partials + ((size_t)par * a.max_blocks + blockIdx.x) * kNQ, sh_red);
        if (flags & F_OPENING) {
            float m = block_max(dmax, sh_f);
            if (threadIdx.x == 0 && m > 0.0f) atomicMax(&ctl->dmax2[stp & 1], __float_as_uint(m));
        }
    }

    __device__ void open_pass(long long stp)
    {
        float dmax = 0.0f;
        for (int i = gt; i < d.n; i += gn) dmax = fmaxf(dmax, open_from_stored(d, a, pc, ac, i, stp));
        float m = block_max(dmax, sh_f);
        if (threadIdx.x == 0 && m > 0.0f) atomicMax(&ctl->dmax2[stp & 1], __float_as_uint(m));
    }

    // Deterministic reduction of one force pass's block partials: block q
    // sums quantity q over all blocks in a fixed order.
    __device__ void reduce_thermo(int par)
    {
        if (blockIdx.x >= kNQ) return;
        double s = 0.0;
        const double* src = d.partials + (size_t)par * a.max_blocks * kNQ + blockIdx.x;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += src[(size_t)b * kNQ];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int lw = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lw == 0) sh_red[w] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x + 31) / 32; k++) t += sh_red[k];
            ctl->thermo[blockIdx.x] = t;
        }
        __syncthreads();
    }

    __device__ void add_disp(long long stp)
    {
        if (threadIdx.x == 0)
            *s_disp += sqrtf(__uint_as_float((unsigned)ld_relaxed((const int*)&ctl->dmax2[stp & 1])));
        __syncthreads();
    }
};

template <typename Real, int LB, bool UNI>
__global__ void __launch_bounds__(kBlock, 1) k_run(Dev<Real> d, RunArgs a)
{
    __shared__ PairP<Real> tab[kMaxTypes * kMaxTypes];
    __shared__ double sh_red[kNQ * 32];
    __shared__ int sh_int[64];
    __shared__ float sh_f[32];
    __shared__ int s_ok;
    __shared__ float s_disp;
    extern __shared__ __align__(32) unsigned char dyn[];

    Ctl* ctl = d.ctl;
    const int ntt = d.ntypes * d.ntypes;
    for (int t = threadIdx.x; t < ntt; t += blockDim.x) tab[t] = d.table[t];
    if (threadIdx.x == 0) s_disp = (float)ctl->disp;

    int state = ctl->state;
    long long step = ctl->step;
    // the list's block partition depends on the grid: rebuild if it changed
    int need_rb = ctl->need_rebuild | a.force_rebuild | (ctl->list_grid != (int)gridDim.x);
    int remaining = a.nsteps;
    int done = 0;
    int parity = 0;
    int have_thermo = 0;
    int rc = 0;  // 0 ok, 1 overflow
    __syncthreads();
    Runner<Real, LB, UNI> R(d, a, tab, sh_red, sh_int, sh_f, &s_ok, &s_disp, dyn);
    R.pc = ctl->pos_cur;
    R.ac = ctl->arr_cur;

    if (a.build_only) {
        rc = R.rebuild();
        if (rc == 2) return;
        need_rb = rc;
    } else {
        if (state == 1) {
            if (need_rb || 2.0f * s_disp > (float)a.skin_eff) {
                rc = R.rebuild();
                if (rc == 2) return;
                need_rb = rc;
            }
            if (rc == 0) {
                R.s_pass();
                if (!R.barrier(10)) return;
                parity = (int)(step & 1);
                R.f_pass(F_STORE, step, parity);
                have_thermo = 1;
                state = 0;
                if (!R.barrier(11)) return;
            }
        }
        if (rc == 0 && remaining > 0 && state == 0) {
            if (threadIdx.x == 0 && blockIdx.x == 0) ctl->dmax2[step & 1] = 0u;
            if (!R.barrier(12)) return;
            R.open_pass(step);
            R.pc ^= 1;
            state = 2;
            if (!R.barrier(13)) return;
            R.add_disp(step);
        }
        while (rc == 0 && state == 2) {
            if (threadIdx.x == 0 && blockIdx.x == 0) ctl->dmax2[(step + 1) & 1] = 0u;
            if (need_rb || 2.0f * s_disp > (float)a.skin_eff) {
                rc = R.rebuild();
                if (rc == 2) return;
                need_rb = rc;
                if (rc) break;
            }
            R.s_pass();
            bar_arrive(ctl, R.bs);
            if (have_thermo) R.reduce_thermo(parity);  // previous pass, overlapped with the wait
            if (!bar_wait(ctl, R.bs, a.timeout_ns, 20, &s_ok)) return;
            const bool more = remaining > 1;
            parity = (int)((step + 1) & 1);
            R.f_pass(F_CLOSING | (more ? F_OPENING : F_STORE), step + 1, parity);
            have_thermo = 1;
            step++;
            remaining--;
            done++;
            if (!R.barrier(21)) return;
            if (more) {
                R.pc ^= 1;
                R.add_disp(step);
            } else {
                state = 0;
            }
        }
    }
    if (have_thermo) R.reduce_thermo(parity);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->state = state;
        ctl->pos_cur = R.pc;
        ctl->arr_cur = R.ac;
        ctl->step = step;
        ctl->disp = s_disp;
        ctl->n_rebuilds += R.rebuilds;
        ctl->steps_done = done;
        ctl->need_rebuild = need_rb;
        if (R.rebuilds > 0) ctl->list_grid = rc == 0 ? (int)gridDim.x : -1;
        if (have_thermo) ctl->thermo[Q_SPARE0] = (double)step;
    }
}

// ---------------------------------------------------------------------------
// Host-exchange kernels (user order <-> slot order).

template <typename Real>
__global__ void k_set_state(Dev<Real> d)
{
    typedef typename Dev<Real>::R4 R4;
    const int n = d.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R4 p;
        Real* pc[3] = {&p.x, &p.y, &p.z};
        for (int c = 0; c < 3; c++) {
            double L = (double)d.Lq[c] * kInvFix;
            double x = d.io[3 * i + c];
            double fl = floor(x / L);
            int im = (int)fl;
            double xw = x - fl * L;
            long long q = __double2ll_rn(xw * kFix);
            if (q >= d.Lq[c]) {
                q -= d.Lq[c];
                im++;
            }
            if (q < 0) {
                q += d.Lq[c];
                im--;
            }
            d.xq[0][c * n + i] = q;
            d.img[0][c * n + i] = im + d.io_int[n + 3 * i + c];
            *pc[c] = fix_to_real(q, Real(0));
        }
        int ty = d.io_int[i];
        p.w = pack_w((i << kTypeBits) | ty, Real(0));
        d.pos[0][i] = p;
        R4 v;
        v.x = (Real)d.io[3 * n + 3 * i + 0];
        v.y = (Real)d.io[3 * n + 3 * i + 1];
        v.z = (Real)d.io[3 * n + 3 * i + 2];
        v.w = (Real)(1.0 / d.io[6 * n + i]);
        d.vel[0][i] = v;
    }
}

template <typename Real>
__global__ void k_get_state(Dev<Real> d, int pc, int ac)
{
    typedef typename Dev<Real>::R4 R4;
    const int n = d.n;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        R4 p = d.pos[pc][q];
        int tag = packed_of(p.w) >> kTypeBits;
        R4 v = d.vel[ac][q];
        for (int c = 0; c < 3; c++) {
            d.io[3 * tag + c] = (double)d.xq[ac][c * n + q] * kInvFix;
            d.io_int[n + 3 * tag + c] = d.img[ac][c * n + q];
        }
        d.io[3 * n + 3 * tag + 0] = (double)v.x;
        d.io[3 * n + 3 * tag + 1] = (double)v.y;
        d.io[3 * n + 3 * tag + 2] = (double)v.z;
        d.io_int[tag] = packed_of(p.w) & ((1 << kTypeBits) - 1);
    }
}

template <typename Real>
__global__ void k_get_forces(Dev<Real> d, int pc)
{
    typedef typename Dev<Real>::R4 R4;
    const int n = d.n;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int tag = packed_of(d.pos[pc][q].w) >> kTypeBits;
        R4 f = d.force[q];
        d.io[3 * tag + 0] = (double)f.x;
        d.io[3 * tag + 1] = (double)f.y;
        d.io[3 * tag + 2] = (double)f.z;
    }
}

template <typename Real>
__global__ void k_get_nlist(Dev<Real> d, int pc, int* rows, int* counts, int width)
{
    const int n = d.n;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int tag = packed_of(d.pos[pc][q].w) >> kTypeBits;
        const int4 inf = d.pinfo[q];
        counts[2 * tag] = inf.y;
        counts[2 * tag + 1] = inf.y + inf.w;
        int* out = rows + (size_t)tag * width;
        int k = 0;
        for (int e = inf.x; e < inf.x + inf.y && k < width; e++, k++)
            out[k] = packed_of(d.pos[pc][d.ent_j[e]].w) >> kTypeBits;
        for (int e = inf.z; e < inf.z + inf.w && k < width; e++, k++)
            out[k] = packed_of(d.pos[pc][d.ent_j[e]].w) >> kTypeBits;
    }
}

}  // namespace swp
