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

template <typename Real>
__device__ __forceinline__ Real ipow(Real b, int e)
{
    Real r = Real(1);
    while (e) {
        if (e & 1) r *= b;
        e >>= 1;
        if (e) b *= b;
    }
    return r;
}

// Eq. 2b at squared distance r2: v and f = -(dv/dr)/r.
template <typename Real>
__device__ __forceinline__ void lj_eval(const PairP<Real>& p, Real r2, Real& v, Real& f)
{
    Real ir2 = Real(1) / r2;
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

// Sums kNQ per-thread accumulators over the block into partials[slot][q].
template <typename Real>
__device__ __forceinline__ void block_thermo(const Real* acc, double* out, double* sh)
{
    // sh: kNQ * 32 doubles
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < kNQ; q++) {
        double v = (double)acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[q * 32 + warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNQ) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += sh[threadIdx.x * 32 + w];
        out[threadIdx.x] = s;
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
__device__ void ph_zero_cells(const Dev<Real>& d, int t, int nt)
{
    for (int c = t; c < d.ncell; c += nt) d.cell_cnt[c] = 0;
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

// Block 0 only.
template <typename Real>
__device__ void ph_scan(const Dev<Real>& d, int* sh)
{
    const int T = blockDim.x;
    const int chunk = (d.ncell + T - 1) / T;
    const int beg = min(threadIdx.x * chunk, d.ncell), end = min(beg + chunk, d.ncell);
    int sum = 0;
    for (int c = beg; c < end; c++) sum += d.cell_cnt[c];
    int total;
    int run = block_excl_scan(sum, sh, &total);
    for (int c = beg; c < end; c++) {
        d.cell_start[c] = run;
        d.cell_fill[c] = run;
        run += d.cell_cnt[c];
    }
    if (threadIdx.x == 0) d.cell_start[d.ncell] = total;
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

// One row per particle: reactive partners first (front), others from the
// back, then moved down behind the reactive block.  Returns the longest row
// seen by this thread.
template <typename Real>
__device__ int ph_build_rows(const Dev<Real>& d, const PairP<Real>* tab, int pc, int t, int nt)
{
    typedef typename Dev<Real>::R4 R4;
    const R4* pos = d.pos[pc];
    const int M = d.max_nn;
    int longest = 0;
    for (int i = t; i < d.n; i += nt) {
        R4 pi = pos[i];
        int ti = type_of(pi);
        int cx, cy, cz;
        cell_coords(d, pi, cx, cy, cz);
        int* row = d.nlist + (size_t)i * M;
        int nr = 0, nw = 0;
        for (int oz = -1; oz <= 1; oz++) {
            int z = cz + oz;
            z = z < 0 ? z + d.nc[2] : (z >= d.nc[2] ? z - d.nc[2] : z);
            for (int oy = -1; oy <= 1; oy++) {
                int y = cy + oy;
                y = y < 0 ? y + d.nc[1] : (y >= d.nc[1] ? y - d.nc[1] : y);
                for (int ox = -1; ox <= 1; ox++) {
                    int x = cx + ox;
                    x = x < 0 ? x + d.nc[0] : (x >= d.nc[0] ? x - d.nc[0] : x);
                    int r = __ldg(&d.cell_rank[(z * d.nc[1] + y) * d.nc[0] + x]);
                    int s = d.cell_start[r], e = d.cell_start[r + 1];
                    for (int q = s; q < e; q++) {
                        if (q == i) continue;
                        R4 pj = pos[q];
                        const PairP<Real>& p = tab[ti * d.ntypes + type_of(pj)];
                        Real dx, dy, dz;
                        Real d2 = dist2(pi, pj, d, dx, dy, dz);
                        if (d2 < p.rlist2) {
                            if (nr + nw < M) {
                                if (p.kind == KIND_SWAP) row[nr] = q;
                                else row[M - 1 - nw] = q;
                            }
                            if (p.kind == KIND_SWAP) nr++;
                            else nw++;
                        }
                    }
                }
            }
        }
        int tot = nr + nw;
        if (tot <= M)
            for (int u = 0; u < nw; u++) row[nr + u] = row[M - nw + u];
        d.ncnt[i] = make_int2(nr, tot);
        longest = max(longest, tot);
    }
    return longest;
}

// ---------------------------------------------------------------------------
// S pass (K-b1): S_i = sum over reactive partners k inside r_cut of a vh(r_ik).

template <typename Real, int LANES>
__device__ __forceinline__ void s_particle(const Dev<Real>& d, const PairP<Real>* tab, int pc,
                                           int i, int lane, unsigned mask)
{
    typedef typename Dev<Real>::R4 R4;
    const R4* pos = d.pos[pc];
    int2 c = d.ncnt[i];
    R4 pi = pos[i];
    const int ti = type_of(pi);
    const int* row = d.nlist + (size_t)i * d.max_nn;
    Real s = Real(0);
    for (int k = lane; k < c.x; k += LANES) {
        int j = row[k];
        R4 pj = pos[j];
        const PairP<Real>& p = tab[ti * d.ntypes + type_of(pj)];
        Real dx, dy, dz;
        Real r2 = dist2(pi, pj, d, dx, dy, dz);
        if (r2 < p.rc2) {
            Real vh = Real(1);
            if (r2 > p.rmin2) {
                Real v, f;
                lj_eval(p, r2, v, f);
                vh = (p.vshift - v) * p.inv_epshat;
            }
            s += p.a * vh;
        }
    }
    s = group_sum<LANES>(s, mask);
    if (lane == 0) d.S[i] = s;
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
    Real q[kNQ];
};

// Adds a displacement to one fixed-point coordinate, wraps it into the box
// (counting the image) and returns the new snapshot coordinate.
template <typename Real>
__device__ __forceinline__ Real advance_fix(const Dev<Real>& d, int ac, int i, int c, Real dx)
{
    const int n = d.n;
    long long q = d.xq[ac][c * n + i] + real_to_fix(dx);
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

// Advances particle i given its force (lane 0 of its group).  Returns the
// squared displacement of this step's drift (0 when not opening).
template <typename Real>
__device__ __forceinline__ float integrate_one(const Dev<Real>& d, const RunArgs& a, int pc,
                                               int ac, int i, Real fx, Real fy, Real fz,
                                               int flags, long long step, Acc<Real>& acc)
{
    typedef typename Dev<Real>::R4 R4;
    R4 v = d.vel[ac][i];
    const Real im = v.w;
    const Real hdt = Real(0.5) * Real(a.dt);
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
            R4 p = d.pos[pc][i];
            unsigned tag = (unsigned)(packed_of(p.w) >> kTypeBits);
            Real z[3];
            normals3(a.seed, step, tag, z);
            const Real c1 = Real(a.c1), sd = Real(a.c2) * sqrt(im);
            v.x = c1 * v.x + sd * z[0];
            v.y = c1 * v.y + sd * z[1];
            v.z = c1 * v.z + sd * z[2];
        }
        ddx += hdt * v.x;
        ddy += hdt * v.y;
        ddz += hdt * v.z;
        disp2 = (float)(ddx * ddx + ddy * ddy + ddz * ddz);
        R4 np;
        np.x = advance_fix(d, ac, i, 0, ddx);
        np.y = advance_fix(d, ac, i, 1, ddy);
        np.z = advance_fix(d, ac, i, 2, ddz);
        np.w = d.pos[pc][i].w;
        d.pos[pc ^ 1][i] = np;
    }
    d.vel[ac][i] = v;
    return disp2;
}

template <typename Real, int LANES>
__device__ __forceinline__ float f_particle(const Dev<Real>& d, const PairP<Real>* tab,
                                            const RunArgs& a, int pc, int ac, int i, int lane,
                                            unsigned mask, int flags, long long step,
                                            Acc<Real>& acc)
{
    typedef typename Dev<Real>::R4 R4;
    const R4* pos = d.pos[pc];
    int2 c = d.ncnt[i];
    R4 pi = pos[i];
    const Real Si = d.S[i];
    const int ti = type_of(pi);
    const int* row = d.nlist + (size_t)i * d.max_nn;
    Real fx = 0, fy = 0, fz = 0;
    for (int k = lane; k < c.x; k += LANES) {  // reactive partners
        int j = row[k];
        R4 pj = pos[j];
        Real Sj = d.S[j];
        const PairP<Real>& p = tab[ti * d.ntypes + type_of(pj)];
        Real dx, dy, dz;
        Real r2 = dist2(pi, pj, d, dx, dy, dz);
        if (r2 < p.rc2) {
            Real v, f2;
            lj_eval(p, r2, v, f2);
            Real ft = f2, vh = Real(1);
            if (r2 > p.rmin2) {
                vh = (p.vshift - v) * p.inv_epshat;
                Real h = p.a * (Si + Sj - Real(2) * p.a * vh);
                ft = f2 * (Real(1) - h * p.inv_epshat);
            }
            acc.q[Q_U2] += Real(0.5) * (v + p.ushift);
            acc.q[Q_U3] += Real(0.5) * p.a * vh * (Si - p.a * vh);
            fx -= ft * dx;
            fy -= ft * dy;
            fz -= ft * dz;
            Real hf = Real(0.5) * ft;
            acc.q[Q_W0 + 0] += hf * dx * dx;
            acc.q[Q_W0 + 1] += hf * dy * dy;
            acc.q[Q_W0 + 2] += hf * dz * dz;
            acc.q[Q_W0 + 3] += hf * dx * dy;
            acc.q[Q_W0 + 4] += hf * dx * dz;
            acc.q[Q_W0 + 5] += hf * dy * dz;
            if (r2 < p.rbond2) acc.q[Q_BONDS] += Real(0.5);
        }
    }
    for (int k = c.x + lane; k < c.y; k += LANES) {  // other pairs (WCA)
        int j = row[k];
        R4 pj = pos[j];
        const PairP<Real>& p = tab[ti * d.ntypes + type_of(pj)];
        Real dx, dy, dz;
        Real r2 = dist2(pi, pj, d, dx, dy, dz);
        if (r2 < p.rc2) {
            Real v, f2;
            lj_eval(p, r2, v, f2);
            acc.q[Q_U2] += Real(0.5) * (v + p.ushift);
            fx -= f2 * dx;
            fy -= f2 * dy;
            fz -= f2 * dz;
            Real hf = Real(0.5) * f2;
            acc.q[Q_W0 + 0] += hf * dx * dx;
            acc.q[Q_W0 + 1] += hf * dy * dy;
            acc.q[Q_W0 + 2] += hf * dz * dz;
            acc.q[Q_W0 + 3] += hf * dx * dy;
            acc.q[Q_W0 + 4] += hf * dx * dz;
            acc.q[Q_W0 + 5] += hf * dy * dz;
        }
    }
    fx = group_sum<LANES>(fx, mask);
    fy = group_sum<LANES>(fy, mask);
    fz = group_sum<LANES>(fz, mask);
    float disp2 = 0.0f;
    if (lane == 0) {
        if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(&d.ctl->status, kStatusNonfinite);
        if (flags & F_STORE) {
            R4 f;
            f.x = fx;
            f.y = fy;
            f.z = fz;
            f.w = Real(0);
            d.force[i] = f;
        }
        disp2 = integrate_one(d, a, pc, ac, i, fx, fy, fz, flags, step, acc);
    }
    return disp2;
}

// Opening half of a step from stored forces (start of a run).
template <typename Real>
__device__ __forceinline__ float open_from_stored(const Dev<Real>& d, const RunArgs& a, int pc,
                                                  int ac, int i, long long step)
{
    typedef typename Dev<Real>::R4 R4;
    R4 f = d.force[i];
    Acc<Real> unused;
#pragma unroll
    for (int q = 0; q < kNQ; q++) unused.q[q] = Real(0);
    return integrate_one(d, a, pc, ac, i, f.x, f.y, f.z, F_OPENING, step, unused);
}

// ---------------------------------------------------------------------------
// The persistent step kernel.  One cooperative launch advances a.nsteps time
// steps (or only rebuilds, or only brings the forces up to date), with two
// grid barriers per step and a rebuild whenever the accumulated displacement
// bound can let an unlisted pair come inside its cut-off.



template <typename Real, int LANES>
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
    Ctl* ctl;
    int gt, gn, lane, gid, ngroups;
    unsigned mask;
    int pc, ac;
    long long rebuilds;
    BarState bs;

    __device__ Runner(const Dev<Real>& d_, const RunArgs& a_, PairP<Real>* tab_, double* sr,
                      int* si, float* sf, int* so, float* sd)
        : d(d_), a(a_), tab(tab_), sh_red(sr), sh_int(si), sh_f(sf), s_ok(so), s_disp(sd),
          ctl(d_.ctl)
    {
        gt = blockIdx.x * blockDim.x + threadIdx.x;
        gn = gridDim.x * blockDim.x;
        lane = gt % LANES;
        gid = gt / LANES;
        ngroups = gn / LANES;
        mask = group_mask<LANES>();
        rebuilds = 0;
        bs.target = 0;
    }

    __device__ __forceinline__ bool barrier(int where)
    {
        bar_arrive(ctl, bs);
        return bar_wait(ctl, bs, a.timeout_ns, where, s_ok);
    }

    // 0: ok; 1: a row overflowed max_nn; 2: a wait timed out.
    __device__ int rebuild()
    {
        if (threadIdx.x == 0 && blockIdx.x == 0) ctl->max_row = 0;
        ph_zero_cells(d, gt, gn);
        if (!barrier(1)) return 2;
        ph_bin(d, pc, gt, gn);
        if (!barrier(2)) return 2;
        if (blockIdx.x == 0) ph_scan(d, sh_int);
        if (!barrier(3)) return 2;
        ph_scatter(d, gt, gn);
        if (!barrier(4)) return 2;
        ph_cell_sort(d, gt, gn);
        if (!barrier(5)) return 2;
        ph_gather(d, pc, ac, gt, gn);
        pc ^= 1;
        ac ^= 1;
        if (!barrier(6)) return 2;
        int longest = ph_build_rows(d, tab, pc, gt, gn);
        int m = block_max_int(longest, sh_int);
        if (threadIdx.x == 0) atomicMax(&ctl->max_row, m);
        if (!barrier(7)) return 2;
        int mr = ld_relaxed(&ctl->max_row);
        rebuilds++;
        if (threadIdx.x == 0) *s_disp = 0.0f;
        __syncthreads();
        if (mr > d.max_nn) {
            if (gt == 0) atomicOr(&ctl->status, kStatusOverflow);
            return 1;
        }
        return 0;
    }

    __device__ void s_pass()
    {
        for (int i = gid; i < d.n; i += ngroups) s_particle<Real, LANES>(d, tab, pc, i, lane, mask);
    }

    __device__ void f_pass(int flags, long long stp, int par)
    {
        Acc<Real> acc;
#pragma unroll
        for (int q = 0; q < kNQ; q++) acc.q[q] = Real(0);
        float dmax = 0.0f;
        for (int i = gid; i < d.n; i += ngroups)
            dmax = fmaxf(dmax, f_particle<Real, LANES>(d, tab, a, pc, ac, i, lane, mask, flags,
                                                       stp, acc));
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

template <typename Real, int LANES>
__global__ void __launch_bounds__(kBlock, 2) k_run(Dev<Real> d, RunArgs a)
{
    __shared__ PairP<Real> tab[kMaxTypes * kMaxTypes];
    __shared__ double sh_red[kNQ * 32];
    __shared__ int sh_int[64];
    __shared__ float sh_f[32];
    __shared__ int s_ok;
    __shared__ float s_disp;

    Ctl* ctl = d.ctl;
    const int ntt = d.ntypes * d.ntypes;
    for (int t = threadIdx.x; t < ntt; t += blockDim.x) tab[t] = d.table[t];
    if (threadIdx.x == 0) s_disp = (float)ctl->disp;

    Runner<Real, LANES> R(d, a, tab, sh_red, sh_int, sh_f, &s_ok, &s_disp);
    int state = ctl->state;
    R.pc = ctl->pos_cur;
    R.ac = ctl->arr_cur;
    long long step = ctl->step;
    int need_rb = ctl->need_rebuild | a.force_rebuild;
    int remaining = a.nsteps;
    int done = 0;
    int parity = 0;
    int have_thermo = 0;
    int rc = 0;  // 0 ok, 1 overflow
    __syncthreads();

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
__global__ void k_get_nlist(Dev<Real> d, int pc, int* rows, int* counts)
{
    const int n = d.n;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int tag = packed_of(d.pos[pc][q].w) >> kTypeBits;
        int2 c = d.ncnt[q];
        counts[2 * tag] = c.x;
        counts[2 * tag + 1] = c.y;
        const int* row = d.nlist + (size_t)q * d.max_nn;
        for (int k = 0; k < c.y && k < d.max_nn; k++)
            rows[(size_t)tag * d.max_nn + k] = packed_of(d.pos[pc][row[k]].w) >> kTypeBits;
    }
}

}  // namespace swp
