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
//
// This file is compiled several times: with SWP_BATCHED 0 into namespace
// swp::single (the single-system step kernel and the exchange kernels; see
// swp_launch.cuh) and with SWP_BATCHED 1 into one namespace per block shape
// of the batched kernel (SWP_BATCH_NS, SWP_BATCH_THREADS threads per block,
// SWP_BATCH_MINB blocks per SM in its launch bounds; see swp_batch_impl.cuh),
// so that the code a group of one block or a group of fewer blocks than
// thermo quantities needs costs the single-system kernel nothing.

#include "swp_internal.h"

#ifndef SWP_BATCHED
#error "define SWP_BATCHED (0 or 1) before including swp_kernels.cuh"
#endif

// With SWP_BATCHED 0 and SWP_WIDE 1 it is compiled into namespace swp::wide:
// the single-system step kernel with 1024-thread blocks (two-barrier step
// only), which bonded networks run: their gathers' latency is hidden better
// with more warps.  That copy leaves out the resident step and the exchange
// kernels.
#undef SWP_HAS_RESIDENT
#if !SWP_BATCHED && !SWP_WIDE
#define SWP_HAS_RESIDENT 1
#else
#define SWP_HAS_RESIDENT 0
#endif

namespace swp {
#if SWP_BATCHED
#if !defined(SWP_BATCH_NS) || !defined(SWP_BATCH_THREADS) || !defined(SWP_BATCH_MINB)
#error "define SWP_BATCH_NS, SWP_BATCH_THREADS and SWP_BATCH_MINB with SWP_BATCHED 1"
#endif
namespace SWP_BATCH_NS {
#elif SWP_WIDE
namespace wide {
#else
namespace single {
#endif

constexpr bool kBatched = SWP_BATCHED != 0;
// The list rebuild is kept out of line in the batched kernel: inlined, its
// register needs spread into the step loop (whose per-system descriptors come
// from shared memory there, not the parameter bank) and cost spills.
#undef SWP_COLD
#if SWP_BATCHED
#define SWP_COLD __noinline__
#else
#define SWP_COLD
#endif
// Threads per block.  The batched kernel reads every system's descriptors from
// shared memory rather than the constant bank; its block shapes trade
// registers per thread (spills at 1024 threads, 64 registers) against warps
// per SM, and SwapBatch.autotune times them on the batch at hand.  The
// single-system kernel runs 768 threads (80 registers): its resident step
// keeps a thread's row, the integrator's state and the pair arithmetic in
// registers at once.
#if SWP_BATCHED
constexpr int kThreads = SWP_BATCH_THREADS;
constexpr int kMinBlocks = SWP_BATCH_MINB;
#elif SWP_WIDE
constexpr int kThreads = kBlockWide;
#else
constexpr int kThreads = kBlock;
#endif

// ---------------------------------------------------------------------------
// Group of blocks that advances one system: the whole grid for a single
// system; in a batched launch, the blocks given to that system (possibly one).
// Every phase partitions its work over the group, and grid barriers are
// barriers over the group.
#if SWP_BATCHED
static __shared__ int s_grp[2];  // [0] this block's rank in the group, [1] group size
__device__ __forceinline__ int g_rank() { return s_grp[0]; }
__device__ __forceinline__ int g_size() { return s_grp[1]; }
#else
__device__ __forceinline__ int g_rank() { return blockIdx.x; }
__device__ __forceinline__ int g_size() { return gridDim.x; }
#endif

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

// Packed tag/type bits of a position snapshot.
__device__ __forceinline__ int pos_bits(const int4& p) { return p.w; }
__device__ __forceinline__ int pos_bits(const dbl4& p) { return packed_of(p.w); }

// Fixed point <-> arithmetic precision.  FP32: through 32-bit halves (the
// 64-bit conversions are slow on this part).  q = hi 2^32 + lo with hi and lo
// converted exactly whenever q carries at most 24 significant bits (every
// float position does), so a float position round-trips exactly; otherwise
// the result is within one float ulp.  The displacement x 2^48 is split at
// 2^24: both halves are exact integers in float for |x| >= 2^-25.
__device__ __forceinline__ float fix_to_real(long long q, float)
{
    const float hi = (float)(int)(q >> 32);
    const float lo = __uint2float_rn((unsigned)(q & 0xffffffffll));
    return fmaf(hi, 0x1p32f, lo) * 0x1p-48f;
}
__device__ __forceinline__ double fix_to_real(long long q, double) { return __ll2double_rn(q) * kInvFix; }
__device__ __forceinline__ long long real_to_fix(float x)
{
    const float y = x * 0x1p24f;
    const float h = truncf(y);
    const int hi = (int)h;
    const int lo = __float2int_rn((y - h) * 0x1p24f);
    return (long long)hi * 16777216ll + lo;
}
__device__ __forceinline__ long long real_to_fix(double x) { return __double2ll_rn(x * kFix); }

__device__ __forceinline__ const PairP<float>* uni_params(const RunArgs& a, float) { return a.uf; }
__device__ __forceinline__ const PairP<double>* uni_params(const RunArgs& a, double) { return a.ud; }

// Selects the run constant of the arithmetic precision.
__device__ __forceinline__ float pick(float, float f, double) { return f; }
__device__ __forceinline__ double pick(double, float, double d) { return d; }

template <typename P4>
__device__ __forceinline__ int type_of(const P4& p) { return pos_bits(p) & ((1 << kTypeBits) - 1); }

// Snapshot coordinate c of fixed-point coordinate q: FP32, the 32-bit box
// fraction floor(q fmul / 2^64); FP64, the coordinate itself.
__device__ __forceinline__ int snap_coord(long long q, int c, const Dev<float>& d)
{
    return (int)__umul64hi((unsigned long long)q, d.fmul[c]);
}
__device__ __forceinline__ double snap_coord(long long q, int, const Dev<double>&) { return fix_to_real(q, 0.0); }
__device__ __forceinline__ int snap_bits(int b, const Dev<float>&) { return b; }
__device__ __forceinline__ double snap_bits(int b, const Dev<double>&) { return pack_w(b, 0.0); }

// FP32 minimum-image displacement of box fractions a -> b along c: the
// wrap-around difference of the fractions (exact), converted and scaled with
// one rounding each.
__device__ __forceinline__ float frac_delta(int a, int b, int c, const Dev<float>& d)
{
    return __fmul_rn(__int2float_rn((int)((unsigned)b - (unsigned)a)), d.fscale[c]);
}

__device__ __forceinline__ float frac_dist2(const int4& pi, const int4& pj, const Dev<float>& d, float& dx,
                                            float& dy, float& dz)
{
    dx = frac_delta(pi.x, pj.x, 0, d);
    dy = frac_delta(pi.y, pj.y, 1, d);
    dz = frac_delta(pi.z, pj.z, 2, d);
    float s = mul_rn(dx, dx);
    s = add_rn(s, mul_rn(dy, dy));
    s = add_rn(s, mul_rn(dz, dz));
    return s;
}

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

// FP32 snapshots: one rule for every distance (the fraction difference is
// already the minimum image).
__device__ __forceinline__ float dist2(const int4& pi, const int4& pj, const Dev<float>& d, float& dx, float& dy,
                                       float& dz)
{
    return frac_dist2(pi, pj, d, dx, dy, dz);
}
__device__ __forceinline__ float dist2_listed(const int4& pi, const int4& pj, const Dev<float>& d, float& dx,
                                              float& dy, float& dz)
{
    return frac_dist2(pi, pj, d, dx, dy, dz);
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

// FP32: the hardware reciprocal approximation (PTX rcp.approx, relative error
// below 2^-22): it feeds only the values of the potential and forces, never a
// decision, and its error is far inside the FP32 force tolerance.
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
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
// FP32: the hardware logarithm and sine/cosine (absolute error about 1e-6 on
// these arguments, far below what the noise amplitude sqrt((1 - c^2) kT/m)
// lets through to a trajectory), at a fifth of the accurate functions' cost.
__device__ __forceinline__ void normals3(unsigned long long seed, long long step, unsigned tag,
                                         float z[3])
{
    uint4 w = philox4x32_10(make_uint4(tag, (unsigned)step, (unsigned)((unsigned long long)step >> 32), 1u),
                            make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const float s32 = 2.3283064365386963e-10f;
    const float two_pi = 6.28318530717958648f;
    float u0 = (__uint2float_rn(w.x) + 0.5f) * s32;
    float u1 = (__uint2float_rn(w.y) + 0.5f) * s32;
    float u2 = (__uint2float_rn(w.z) + 0.5f) * s32;
    float u3 = (__uint2float_rn(w.w) + 0.5f) * s32;
    float ra = sqrtf(-2.0f * __logf(u0));
    float rb = sqrtf(-2.0f * __logf(u2));
    float sn, cs;
    __sincosf(two_pi * u1, &sn, &cs);
    z[0] = ra * cs;
    z[1] = ra * sn;
    z[2] = rb * __cosf(two_pi * u3);
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

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Set (thread 0 of one block) when the launch must withhold that block's
// arrival at its first grid barrier (a test of the bounded waits).
static __shared__ int s_withhold;

// Arrival: the block's writes are ordered before a release add on the
// counter (after the block-wide __syncthreads, thread 0's release is
// cumulative over them).  Generation g completes at count g * (group size).
// With pub_dst set, thread 0 first folds the block's shared maximum *pub_src
// into the global maximum *pub_dst (and clears it), so the other blocks see
// it after their wait.
__device__ __forceinline__ void bar_arrive(Ctl* ctl, BarState& b, unsigned* pub_dst = nullptr,
                                           unsigned* pub_src = nullptr)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        if (pub_dst) {
            const unsigned m = *pub_src;
            if (m) atomicMax(pub_dst, m);
            *pub_src = 0u;
        }
        if (kBatched && g_size() == 1) return;  // a group of one block: __syncthreads is the barrier
        b.target += g_size();
        if (s_withhold)
            s_withhold = 0;  // this arrival is withheld: every wait of the barrier runs out
        else
            asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(&ctl->barrier), "l"(1ull) : "memory");
    }
}

// Wait: acquire polling, bounded in time.  Every arrival is a release add on
// the counter, and later adds continue its release sequence, so the load that
// first sees the target synchronises with every arrival: the other blocks'
// writes are visible to this block after the __syncthreads.  (Relaxed polling
// followed by an acquire fence measured 0.4 us slower per step.)
__device__ __forceinline__ bool bar_wait(Ctl* ctl, const BarState& b, long long timeout_ns,
                                         int where, int* s_ok)
{
    if (kBatched && g_size() == 1) {
        __syncthreads();
        return true;
    }
    if (threadIdx.x == 0) {
        int ok = 1;
        int spins = 0;
        long long t0 = 0;
        while (ld_acquire_u64(&ctl->barrier) < b.target) {
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
            __nanosleep(32);
        }
        *s_ok = ok;
    }
    __syncthreads();
    if (*s_ok == 0) asm volatile("cp.async.wait_all;" ::: "memory");  // leave no copy in flight
    return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Block reductions

// Compensated FP32 summation (Knuth's TwoSum; the double-float addition of
// Dekker and Bailey): a pair (hi, lo) carries about 44 significant bits, so
// the block sums below lose nothing beyond the per-thread FP32 terms.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl)
{
    float s, e;
    two_sum(hi, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// Block sums of the per-thread thermo accumulators (energies, virial, bond
// count), added to the block's FP64 running sums blk[q]; with out given,
// blk[q] is then written to out[q] (the block's partial of the pass) and
// cleared.  Each thread holds the terms of one sub-chunk at most (multi-chunk
// passes flush after every sub-chunk), so the error does not grow with the
// system size; block partials are summed over blocks in FP64
// (run_reduce_thermo).
//
// FP32 runs: each warp folds its lanes' values by a shuffle tree (at most five
// roundings of the warp's sum of magnitudes) into s_wpart[q][warp]; warp q
// then sums quantity q over the block's warps compensated (double-float).
// FP64 runs: the values are staged in shared memory (stage: kNQA x blockDim)
// and warp q sums them in FP64.
static __shared__ float s_wpart[kNQA][32];

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// s_wpart[q][warp] = the warp's sum of x (every lane of the warp calls it).
__device__ __forceinline__ void warp_part(float x, int q)
{
    x = warp_sum(x);
    if ((threadIdx.x & 31) == 0) s_wpart[q][threadIdx.x >> 5] = x;
}

// Sums s_wpart over the block's warps into blk / out (see above); out2, when
// given with out, gets the same values.  The caller orders the s_wpart writes
// before and the next ones after (block_sums_from_warps: two __syncthreads).
__device__ __forceinline__ void warp_sums_to(double* blk, double* out, double* out2)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int q = warp; q < kNQ; q += nw) {  // quantity q by warp q mod nw (blocks of fewer warps)
        if (q >= kNQA) {
            if (out && lane == 0) {
                out[q] = 0.0;
                if (out2) out2[q] = 0.0;
            }
            continue;
        }
        float hi = lane < nw ? s_wpart[q][lane] : 0.0f, lo = 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            df_add(hi, lo, h2, l2);
        }
        if (lane == 0) {
            const double tot = blk[q] + ((double)hi + (double)lo);
            if (out) {
                out[q] = tot;
                if (out2) out2[q] = tot;
                blk[q] = 0.0;
            } else {
                blk[q] = tot;
            }
        }
    }
}

__device__ __forceinline__ void block_sums_from_warps(double* blk, double* out, double* out2 = nullptr)
{
    __syncthreads();
    warp_sums_to(blk, out, out2);
    __syncthreads();
}

__device__ __forceinline__ void block_sums(const float* acc, float*, double* blk, double* out,
                                           double* out2 = nullptr)
{
#pragma unroll
    for (int q = 0; q < kNQA; q++) warp_part(acc[q], q);
    block_sums_from_warps(blk, out, out2);
}

__device__ __forceinline__ void block_sums(const double* acc, double* stage, double* blk, double* out,
                                           double* out2 = nullptr)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, B = blockDim.x, nw = (B + 31) >> 5;
#pragma unroll
    for (int q = 0; q < kNQA; q++) stage[q * B + t] = acc[q];
    __syncthreads();
    for (int q = warp; q < kNQ; q += nw) {  // quantity q by warp q mod nw
        if (q >= kNQA) {
            if (out && lane == 0) {
                out[q] = 0.0;
                if (out2) out2[q] = 0.0;
            }
            continue;
        }
        double x = 0.0;
        for (int k = lane; k < B; k += 32) x += stage[q * B + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) {
            const double tot = blk[q] + x;
            if (out) {
                out[q] = tot;
                if (out2) out2[q] = tot;
                blk[q] = 0.0;
            } else {
                blk[q] = tot;
            }
        }
    }
    __syncthreads();
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
// Neighbour-list rebuild phases: bin by cell, counting sort with a
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

// FP32 snapshots: the cell of a box fraction u is floor(u nc / 2^32), exact.
__device__ __forceinline__ void cell_coords(const Dev<float>& d, const int4& p, int& cx, int& cy, int& cz)
{
    cx = min((int)__umulhi((unsigned)p.x, (unsigned)d.nc[0]), d.nc[0] - 1);
    cy = min((int)__umulhi((unsigned)p.y, (unsigned)d.nc[1]), d.nc[1] - 1);
    cz = min((int)__umulhi((unsigned)p.z, (unsigned)d.nc[2]), d.nc[2] - 1);
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
    const int ch = (d.ncell + g_size() - 1) / g_size();
    const int beg = min(g_rank() * ch, d.ncell), end = min(beg + ch, d.ncell);
    int v = 0;
    for (int c = beg + threadIdx.x; c < end; c += blockDim.x) v += d.cell_cnt[c];
    int t = block_sum_int(v, sh);
    if (threadIdx.x == 0) d.bsum[g_rank()] = t;
}

template <typename Real>
__device__ void ph_chunk_scan(const Dev<Real>& d, int* sh)
{
    const int ch = (d.ncell + g_size() - 1) / g_size();
    const int beg = min(g_rank() * ch, d.ncell), end = min(beg + ch, d.ncell);
    int v = 0;
    for (int b = threadIdx.x; b < g_rank(); b += blockDim.x) v += d.bsum[b];
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
        const typename Dev<Real>::P4 pp = d.pos[pc][p];
        d.pos[pc ^ 1][q] = pp;
        if (d.has_bonds) d.slot_of_tag[pos_bits(pp) >> kTypeBits] = q;
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
    const int Pb = (d.n + g_size() - 1) / g_size();
    b0 = min(g_rank() * Pb, d.n);
    b1 = min(b0 + Pb, d.n);
}

// Builds the block's entries (last rebuild phase), one warp per cell: the warp
// loads the 27 stencil ranges of its cell once, then tests its member
// particles against the candidates 32 at a time with warp ballots.  A
// counting sweep, a block scan that places every particle's runs (reactive
// entries of the sub-chunk first, then the others), and a writing sweep;
// candidates keep the stencil order, so the output is deterministic.
// cnt: blockDim.x int2 of shared memory.  Returns the block's entry count
// per particle (rounded up), the row length a capacity check needs.
template <typename Real>
__device__ __forceinline__ int rank_of(const Dev<Real>& d, const typename Dev<Real>::P4& p)
{
    int cx, cy, cz;
    cell_coords(d, p, cx, cy, cz);
    return __ldg(&d.cell_rank[(cz * d.nc[1] + cy) * d.nc[0] + cx]);
}

template <typename Real>
__device__ int ph_build_cells(const Dev<Real>& d, const PairP<Real>* tab, int pc, int2* cnt,
                              int* sh, int* overflow)
{
    typedef typename Dev<Real>::P4 P4;
    constexpr int NCH = 4;  // candidate chunks of 32 held at once
    const P4* pos = d.pos[pc];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int b0, b1;
    block_range(d, b0, b1);
    const int Pb = (d.n + g_size() - 1) / g_size();
    const long long cap_beg = (long long)g_rank() * Pb * d.max_nn;
    const long long cap_end = cap_beg + (long long)Pb * d.max_nn;
    long long base = cap_beg;
    for (int q0 = b0; q0 < b1; q0 += blockDim.x) {
        const int q1 = min(q0 + (int)blockDim.x, b1);
        const int P = q1 - q0;
        const int r_lo = rank_of(d, pos[q0]);
        const int r_hi = rank_of(d, pos[q1 - 1]);
        if ((int)threadIdx.x < P) cnt[threadIdx.x] = make_int2(0, 0);
        __syncthreads();
        bool fits = true;
        for (int pass = 0; pass < 2; pass++) {
            if (pass == 1) {
                // place the runs: reactive entries of the sub-chunk, then the others
                const int t = threadIdx.x;
                const int2 c = t < P ? cnt[t] : make_int2(0, 0);
                int Er, Ew;
                const int offr = block_excl_scan(c.x, sh, &Er);
                const int offw = block_excl_scan(c.y, sh, &Ew);
                fits = base + Er + Ew <= cap_end;
                if (t < P) {
                    const int ro = (int)(base + offr), wo = (int)(base + Er + offw);
                    d.pinfo[q0 + t] = make_int4(ro, c.x, wo, c.y);
                    cnt[t] = make_int2(ro, wo);  // running write positions
                }
                if (!fits && t == 0) *overflow = 1;
                base += Er + Ew;
                __syncthreads();
                if (!fits) break;
            }
            for (int r = r_lo + warp; r <= r_hi; r += nwarps) {
                const int m0 = max(d.cell_start[r], q0), m1 = min(d.cell_start[r + 1], q1);
                if (m0 >= m1) continue;
                // the 27 stencil ranges (lane l < 27 holds range l)
                const int lin = __ldg(&d.cell_rank[d.ncell + r]);
                const int cx = lin % d.nc[0], cy = (lin / d.nc[0]) % d.nc[1], cz = lin / (d.nc[0] * d.nc[1]);
                int s = 0, len = 0;
                if (lane < 27) {
                    int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
                    x = x < 0 ? x + d.nc[0] : (x >= d.nc[0] ? x - d.nc[0] : x);
                    y = y < 0 ? y + d.nc[1] : (y >= d.nc[1] ? y - d.nc[1] : y);
                    z = z < 0 ? z + d.nc[2] : (z >= d.nc[2] ? z - d.nc[2] : z);
                    const int rr = __ldg(&d.cell_rank[(z * d.nc[1] + y) * d.nc[0] + x]);
                    s = d.cell_start[rr];
                    len = d.cell_start[rr + 1] - s;
                }
                int pre = len;  // inclusive prefix over the lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += y;
                }
                const int C = __shfl_sync(0xffffffffu, pre, 31);
                for (int g0 = 0; g0 < C; g0 += 32 * NCH) {
                    // this group's candidates: slot and position per lane and chunk.
                    // Candidate tc lies in the range idx = number of ranges that end
                    // at or before it; every lane runs every shuffle (no divergence).
                    int cq[NCH];
                    P4 cp[NCH];
                    int idx[NCH];
#pragma unroll
                    for (int k = 0; k < NCH; k++) idx[k] = 0;
                    for (int l = 0; l < 27; l++) {
                        const int pl = __shfl_sync(0xffffffffu, pre, l);
#pragma unroll
                        for (int k = 0; k < NCH; k++) idx[k] += (pl <= g0 + 32 * k + lane) ? 1 : 0;
                    }
#pragma unroll
                    for (int k = 0; k < NCH; k++) {
                        const int tc = g0 + 32 * k + lane;
                        const int rg = min(idx[k], 26);
                        const int sl = __shfl_sync(0xffffffffu, s, rg);
                        const int pb = __shfl_sync(0xffffffffu, pre - len, rg);
                        cq[k] = tc < C ? sl + (tc - pb) : -1;
                    }
#pragma unroll
                    for (int k = 0; k < NCH; k++)
                        if (cq[k] >= 0) cp[k] = pos[cq[k]];
                    for (int i = m0; i < m1; i++) {
                        const P4 pi = pos[i];
                        const int ti = type_of(pi);
                        int2 run = cnt[i - q0];
#pragma unroll
                        for (int k = 0; k < NCH; k++) {
                            bool react = false, other = false;
                            if (cq[k] >= 0 && cq[k] != i) {
                                const PairP<Real>& p = tab[ti * d.ntypes + type_of(cp[k])];
                                Real dx, dy, dz;
                                if (dist2(pi, cp[k], d, dx, dy, dz) < p.rlist2) {
                                    react = p.kind == KIND_SWAP;
                                    other = !react;
                                }
                            }
                            const unsigned br = __ballot_sync(0xffffffffu, react);
                            const unsigned bw = __ballot_sync(0xffffffffu, other);
                            if (pass == 1) {
                                if (react) {
                                    const int e = run.x + __popc(br & lt);
                                    d.ent_j[e] = cq[k];
                                    d.ent_o[e] = (unsigned short)(i - q0);
                                }
                                if (other) {
                                    const int e = run.y + __popc(bw & lt);
                                    d.ent_j[e] = cq[k];
                                    d.ent_o[e] = (unsigned short)(i - q0);
                                }
                            }
                            run.x += __popc(br);
                            run.y += __popc(bw);
                        }
                        __syncwarp();
                        if (lane == 0) cnt[i - q0] = run;
                        __syncwarp();
                    }
                }
            }
            __syncthreads();
        }
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

// Shared-memory staging of one sub-chunk (dynamic shared memory): the
// sub-chunk's own particles and the per-entry results of one wave.  The
// regions sit at compile-time offsets from one namespace-scope extern
// __shared__ array, so every access is a direct shared-memory access.
extern __shared__ __align__(32) unsigned char g_dyn[];

template <typename Real>
struct Stage {
    typedef typename Dev<Real>::R4 R4;
    typedef typename Dev<Real>::P4 P4;
    // entries per wave: 8 (FP32) or 3 (FP64) per thread of a batched block shape
    static constexpr int kWave = kBatched ? (sizeof(Real) == 4 ? 8 : 3) * kThreads : (sizeof(Real) == 4 ? 8192 : 3072);
    static constexpr size_t B = kThreads;
    static constexpr size_t O_POS = 0;                                  // [B] P4 positions
    static constexpr size_t O_VEL = O_POS + B * sizeof(P4);             // [B] R4 velocities
    static constexpr size_t O_XQ = O_VEL + B * sizeof(R4);              // [3B] fixed-point positions
    static constexpr size_t O_INFO = O_XQ + 3 * B * sizeof(long long);  // [B] int4 pinfo
    static constexpr size_t O_S = O_INFO + B * sizeof(int4);            // [B] S
    static constexpr size_t O_W = O_S + B * sizeof(Real);               // [kWave] R4 entry results
    static constexpr size_t kBytes = O_W + (size_t)kWave * sizeof(R4);
    static size_t bytes(int) { return kBytes; }

    static __device__ __forceinline__ P4* pos() { return (P4*)(g_dyn + O_POS); }
    static __device__ __forceinline__ R4* vel() { return (R4*)(g_dyn + O_VEL); }
    static __device__ __forceinline__ long long* xq() { return (long long*)(g_dyn + O_XQ); }
    static __device__ __forceinline__ int4* info() { return (int4*)(g_dyn + O_INFO); }
    static __device__ __forceinline__ Real* S() { return (Real*)(g_dyn + O_S); }
    static __device__ __forceinline__ Real* w() { return (Real*)(g_dyn + O_W); }
    static __device__ __forceinline__ R4* w4() { return (R4*)(g_dyn + O_W); }
    static constexpr int wave = kWave;
};

// Asynchronous global -> shared copies (no register staging).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
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
// S pass: S_i = sum over reactive partners k inside r_cut of a vh(r_ik).

// One reactive entry's term of S_i: a vh(r_ij) inside r_cut, else 0 (evaluated
// for every listed pair and selected by the cut-off decision, see entry_force).
template <typename Real, bool UNI>
__device__ __forceinline__ Real s_term(const Dev<Real>& d, const PairP<Real>* tab, const PairP<Real>& ps,
                                       const typename Dev<Real>::P4& pi, const typename Dev<Real>::P4& pj)
{
    const PairP<Real>& p = pair_of<Real, UNI>(tab, type_of(pi), type_of(pj), d.ntypes, ps);
    Real dx, dy, dz;
    const Real r2 = dist2_listed(pi, pj, d, dx, dy, dz);
    Real v, f;
    lj_eval(p, r2, v, f);
    const Real vh = r2 > p.rmin2 ? (p.vshift - v) * p.inv_epshat : Real(1);
    return r2 < p.rc2 ? mul_rn(p.a, vh) : Real(0);
}

// End of the block's region of the list (entries of its particles are
// placed inside [rank * Pb * max_nn, (rank + 1) * Pb * max_nn)).
template <typename Real>
__device__ __forceinline__ long long block_list_end(const Dev<Real>& d)
{
    const long long Pb = (d.n + g_size() - 1) / g_size();
    return (long long)(g_rank() + 1) * Pb * d.max_nn;
}

// Brings list entries [e0, e1) (partner slots and owner indices) into L2, one
// 128-byte line per thread, while the block works on other entries.
template <typename Real>
__device__ __forceinline__ void prefetch_entries(const Dev<Real>& d, long long e0, long long e1)
{
    if (e1 <= e0) return;
    const long long nj = ((e1 - 1) >> 5) - (e0 >> 5) + 1;  // 32 partner slots per line
    const long long no = ((e1 - 1) >> 6) - (e0 >> 6) + 1;  // 64 owner indices per line
    for (long long k = threadIdx.x; k < nj + no; k += blockDim.x) {
        const void* p = k < nj ? (const void*)&d.ent_j[max(((e0 >> 5) + k) << 5, e0)]
                               : (const void*)&d.ent_o[max(((e0 >> 6) + k - nj) << 6, e0)];
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

// Entries per thread whose gathers a two-barrier pass issues together (S
// pass, force pass).
constexpr int kGather = 4;
constexpr int kGatherF = 2;

// staged: the block has one sub-chunk and the shared copies of its positions
// and list ranges are current (kept by the previous force pass), so they are
// not loaded again.  With one sub-chunk the block's S values also stay in
// shared memory for the force pass.
template <typename Real, bool UNI>
__device__ void s_pass_block(const Dev<Real>& d, const PairP<Real>* tab, int pc,
                             const PairP<Real>& ps, bool staged)
{
    typedef Stage<Real> SM;
    typedef typename Dev<Real>::P4 P4;
    const P4* pos = d.pos[pc];
    int b0, b1;
    block_range(d, b0, b1);
    const int t = threadIdx.x;
    const bool single = b1 - b0 <= (int)blockDim.x;
    for (int q0 = b0; q0 < b1; q0 += blockDim.x) {
        const int P = min((int)blockDim.x, b1 - q0);
        if (!staged) {
            if (t < P) {
                SM::pos()[t] = pos[q0 + t];
                SM::info()[t] = d.pinfo[q0 + t];
            }
            __syncthreads();
        }
        const int e_beg = SM::info()[0].x;
        const int e_end = SM::info()[P - 1].x + SM::info()[P - 1].y;
        {
            // into L2 while this sub-chunk runs: the next sub-chunk's reactive
            // entries (sized like this one's), or after the last one the
            // block's first sub-chunk, which the force pass starts with
            const int4 last = SM::info()[P - 1];
            const long long full = (long long)last.z + last.w;
            const long long cap = block_list_end(d);
            if (q0 + P < b1)
                prefetch_entries(d, full, min(full + (e_end - e_beg), cap));
            else {
                const long long f0 = cap - (long long)((d.n + g_size() - 1) / g_size()) * d.max_nn;
                prefetch_entries(d, f0, min(f0 + (full - e_beg), cap));
            }
        }
        Real s = Real(0);
        for (int wb = e_beg; wb < e_end; wb += SM::wave) {
            const int we = min(wb + SM::wave, e_end);
            // the thread's entries e, e + B, ... in groups of kGather: the group's
            // index loads, then its partner gathers, are independent of one
            // another, so that many are in flight when the partners come from DRAM
            const int B = blockDim.x;
            for (int e0 = wb + t; e0 < we; e0 += kGather * B) {
                int jj[kGather], oo[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    const int e = e0 + u * B;
                    jj[u] = e < we ? __ldcs(&d.ent_j[e]) : 0;  // streamed: keep L2 for the snapshots
                    oo[u] = e < we ? __ldcs(&d.ent_o[e]) : 0;
                }
                P4 pp[kGather];
#pragma unroll
                for (int u = 0; u < kGather; u++) pp[u] = pos[jj[u]];  // slot 0 for a missing entry
#pragma unroll
                for (int u = 0; u < kGather; u++) {
                    const int e = e0 + u * B;
                    if (e < we) SM::w()[e - wb] = s_term<Real, UNI>(d, tab, ps, SM::pos()[oo[u]], pp[u]);
                }
            }
            __syncthreads();
            if (t < P) {
                const int4 inf = SM::info()[t];
                const int k0 = max(inf.x, wb), k1 = min(inf.x + inf.y, we);
                int k = k0;
                for (; k + 4 <= k1; k += 4) s += (SM::w()[k - wb] + SM::w()[k + 1 - wb]) + (SM::w()[k + 2 - wb] + SM::w()[k + 3 - wb]);
                for (; k < k1; k++) s += SM::w()[k - wb];
            }
            __syncthreads();
        }
        if (t < P) {
            d.S[q0 + t] = s;
            if (single) SM::S()[t] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Force pass fused with the integrator.
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

// Adds a displacement to one fixed-point coordinate and wraps it into the box;
// w gets the change of the image count (-1, 0 or +1).
__device__ __forceinline__ long long advance_fix(long long q0, long long Lq, long long dq, int& w)
{
    const long long q = q0 + dq;
    if (q >= Lq) {
        w = 1;
        return q - Lq;
    }
    if (q < 0) {
        w = -1;
        return q + Lq;
    }
    w = 0;
    return q;
}

// The integrator on one particle's registers: the closing half kick of the
// step that ends, the kinetic energy, and (opening) the half kick, half drift,
// Langevin O step and half drift of the next (BAOAB; velocity Verlet without
// O).  q[] (fixed point) and v are advanced in place, w[] gets the image
// changes, np the new snapshot.  Returns the squared displacement of the drift
// (0 when not opening).
template <typename Real>
__device__ __forceinline__ float advance_particle(const Dev<Real>& d, const RunArgs& a, Real fx, Real fy, Real fz,
                                                  int flags, long long step, int wbits,
                                                  typename Dev<Real>::R4& v, long long q[3], int w[3], Real& kin,
                                                  typename Dev<Real>::P4& np)
{
    const Real im = v.w;
    const Real hdt = pick(Real(0), a.hdt_f, a.hdt_d);
    if (flags & F_CLOSING) {
        v.x += hdt * fx * im;
        v.y += hdt * fy * im;
        v.z += hdt * fz * im;
    }
    kin += Real(0.5) * (v.x * v.x + v.y * v.y + v.z * v.z) * recip(im);
    float disp2 = 0.0f;
    w[0] = w[1] = w[2] = 0;
    if (flags & F_OPENING) {
        v.x += hdt * fx * im;
        v.y += hdt * fy * im;
        v.z += hdt * fz * im;
        Real ddx = hdt * v.x, ddy = hdt * v.y, ddz = hdt * v.z;
        if (a.langevin) {
            Real z[3];
            normals3(a.seed, step, (unsigned)(wbits >> kTypeBits), z);
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
        q[0] = advance_fix(q[0], d.Lq[0], real_to_fix(ddx), w[0]);
        q[1] = advance_fix(q[1], d.Lq[1], real_to_fix(ddy), w[1]);
        q[2] = advance_fix(q[2], d.Lq[2], real_to_fix(ddz), w[2]);
        np.x = snap_coord(q[0], 0, d);
        np.y = snap_coord(q[1], 1, d);
        np.z = snap_coord(q[2], 2, d);
        np.w = snap_bits(wbits, d);
    }
    return disp2;
}

// Advances particle i given its force (state from global memory, written
// back there; the image count is touched only when the particle wraps).
// Returns the squared displacement of this step's drift (0 when not opening).
template <typename Real>
__device__ __forceinline__ float integrate_one(const Dev<Real>& d, const RunArgs& a, int pc,
                                               int ac, int i, Real fx, Real fy, Real fz,
                                               int flags, long long step, PState<Real>& st,
                                               int wbits, Real& kin, typename Dev<Real>::P4* keep)
{
    typename Dev<Real>::R4 v = st.v;
    typename Dev<Real>::P4 np;
    int w[3];
    const float disp2 = advance_particle(d, a, fx, fy, fz, flags, step, wbits, v, st.q, w, kin, np);
    if (flags & F_OPENING) {
        const int n = d.n;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            __stcs(&d.xq[ac][c * n + i], st.q[c]);  // read again only next step: evict first
            if (w[c]) d.img[ac][c * n + i] += w[c];
        }
        d.pos[pc ^ 1][i] = np;
        if (keep) *keep = np;
    }
    if constexpr (sizeof(Real) == 4)
        __stcs((float4*)&d.vel[ac][i], *(const float4*)&v);
    else
        d.vel[ac][i] = v;
    return disp2;
}

// One entry's pair force on its owner (returned as the components of
// f (x_i - x_j)), with the entry's share of energies, virial and bond count
// when TH (the sampled step of a launch).  REACT: a reactive pair (two-body
// plus the three-body factor); else a purely two-body pair.
template <typename Real, bool UNI, bool REACT, bool TH>
__device__ __forceinline__ void entry_force(const Dev<Real>& d, const PairP<Real>* tab,
                                            const typename Dev<Real>::P4& pi,
                                            const typename Dev<Real>::P4& pj, Real Si, Real Sj,
                                            const PairP<Real>& pu, Acc<Real>& acc, Real& fx,
                                            Real& fy, Real& fz)
{
    Real dx, dy, dz;
    const Real r2 = dist2_listed(pi, pj, d, dx, dy, dz);
    const PairP<Real>& p = pair_of<Real, UNI>(tab, type_of(pi), type_of(pj), d.ntypes, pu);
    // evaluated for every listed pair and selected by the cut-off decision
    // (no divergent branch: about half of the listed pairs lie in the skin)
    const bool in = r2 < p.rc2;
    Real v, ft;
    lj_eval(p, r2, v, ft);
    if (TH) acc.q[Q_U2] += in ? Real(0.5) * (v + p.ushift) : Real(0);
    if (REACT) {
        const bool beyond = r2 > p.rmin2;
        const Real vh = beyond ? (p.vshift - v) * p.inv_epshat : Real(1);
        const Real h = p.a * (Si + Sj - Real(2) * p.a * vh);
        ft = beyond ? ft * (Real(1) - h * p.inv_epshat) : ft;
        if (TH) {
            acc.q[Q_U3] += in ? Real(0.5) * p.a * vh * (Si - p.a * vh) : Real(0);
            acc.q[Q_BONDS] += (in && r2 < p.rbond2) ? Real(0.5) : Real(0);
        }
    }
    ft = in ? ft : Real(0);
    fx = -ft * dx;
    fy = -ft * dy;
    fz = -ft * dz;
    if (!TH) return;
    const Real hf = Real(0.5) * ft;
    acc.q[Q_W0 + 0] += hf * dx * dx;
    acc.q[Q_W0 + 1] += hf * dy * dy;
    acc.q[Q_W0 + 2] += hf * dz * dz;
    acc.q[Q_W0 + 3] += hf * dx * dy;
    acc.q[Q_W0 + 4] += hf * dx * dz;
    acc.q[Q_W0 + 5] += hf * dy * dz;
}

// Adds the per-entry forces w[k - wb] (one vector load each) of entries
// [k0, k1) to f in entry order (the result does not depend on the launch).
template <typename Real, typename R4>
__device__ __forceinline__ void sum_run(const R4* w, int wb, int k0, int k1, Real& fx, Real& fy,
                                        Real& fz)
{
#pragma unroll 2
    for (int k = k0; k < k1; k++) {
        const R4 p = w[k - wb];
        fx += p.x;
        fy += p.y;
        fz += p.z;
    }
}

// With one sub-chunk per block the S pass of the same step left the block's
// positions, list ranges and S values in shared memory, and the integrator
// keeps the shared positions current for the next S pass.  TH: the sampled
// step (thermo terms summed into the block's running sums blk).
template <typename Real, bool UNI, bool BONDS, bool TH>
__device__ float f_pass_block(const Dev<Real>& d, const PairP<Real>* tab, const RunArgs& a, int pc,
                              int ac, int flags, long long step, Acc<Real>& acc,
                              const PairP<Real>& ps, const PairP<Real>& pw, double* blk)
{
    typedef Stage<Real> SM;
    typedef typename Dev<Real>::R4 R4;
    typedef typename Dev<Real>::P4 P4;
    const P4* pos = d.pos[pc];
    int b0, b1;
    block_range(d, b0, b1);
    const int t = threadIdx.x;
    const int n = d.n;
    const bool single = b1 - b0 <= (int)blockDim.x;
    float dmax = 0.0f;
    for (int q0 = b0; q0 < b1; q0 += blockDim.x) {
        const int P = min((int)blockDim.x, b1 - q0);
        if (t < P) {
            const int i = q0 + t;
            // integrator inputs: asynchronous copies, waited for after the entries
            cp_async_r4(&SM::vel()[t], &d.vel[ac][i]);
            if (flags & F_OPENING)
                for (int c = 0; c < 3; c++) cp_async(&SM::xq()[3 * t + c], &d.xq[ac][c * n + i], 8);
            cp_async_commit();
        }
        if (!single) {
            if (t < P) {
                const int i = q0 + t;
                SM::pos()[t] = pos[i];
                SM::S()[t] = d.S[i];
                SM::info()[t] = d.pinfo[i];
            }
            __syncthreads();
        }
        const int e_beg = SM::info()[0].x;
        const int e_rend = SM::info()[P - 1].x + SM::info()[P - 1].y;
        const int e_end = SM::info()[P - 1].z + SM::info()[P - 1].w;
        {
            // into L2 while this sub-chunk runs: the next sub-chunk's entries
            // (sized like this one's), or after the last one the reactive
            // entries of the block's first sub-chunk, which the next S pass
            // starts with
            const long long cap = block_list_end(d);
            if (q0 + P < b1)
                prefetch_entries(d, e_end, min((long long)e_end + (e_end - e_beg), cap));
            else {
                const long long f0 = cap - (long long)((d.n + g_size() - 1) / g_size()) * d.max_nn;
                prefetch_entries(d, f0, min(f0 + (e_rend - e_beg), cap));
            }
        }
        Real fx = 0, fy = 0, fz = 0, gx = 0, gy = 0, gz = 0;  // reactive and other entries' sums
        for (int wb = e_beg; wb < e_end; wb += SM::wave) {
            const int we = min(wb + SM::wave, e_end);
            // groups of kGatherF entries per thread, their gathers issued together
            const int B = blockDim.x;
            for (int e0 = wb + t; e0 < we; e0 += kGatherF * B) {
                int jj[kGatherF], oo[kGatherF];
#pragma unroll
                for (int u = 0; u < kGatherF; u++) {
                    const int e = e0 + u * B;
                    jj[u] = e < we ? __ldcs(&d.ent_j[e]) : 0;  // streamed: keep L2 for the snapshots
                    oo[u] = e < we ? __ldcs(&d.ent_o[e]) : 0;
                }
                P4 pj[kGatherF];
                Real sj[kGatherF];
#pragma unroll
                for (int u = 0; u < kGatherF; u++) {
                    pj[u] = pos[jj[u]];  // slot 0 for a missing entry
                    sj[u] = e0 + u * B < e_rend ? d.S[jj[u]] : Real(0);
                }
#pragma unroll
                for (int u = 0; u < kGatherF; u++) {
                    const int e = e0 + u * B;
                    if (e >= we) continue;
                    Real ex, ey, ez;
                    if (e < e_rend)
                        entry_force<Real, UNI, true, TH>(d, tab, SM::pos()[oo[u]], pj[u], SM::S()[oo[u]], sj[u], ps,
                                                         acc, ex, ey, ez);
                    else
                        entry_force<Real, UNI, false, TH>(d, tab, SM::pos()[oo[u]], pj[u], Real(0), Real(0), pw, acc,
                                                          ex, ey, ez);
                    R4 r;
                    r.x = ex;
                    r.y = ey;
                    r.z = ez;
                    r.w = Real(0);
                    SM::w4()[e - wb] = r;
                }
            }
            __syncthreads();
            if (t < P) {
                const int4 inf = SM::info()[t];
                sum_run(SM::w4(), wb, max(inf.x, wb), min(inf.x + inf.y, we), fx, fy, fz);
                sum_run(SM::w4(), wb, max(inf.z, wb), min(inf.z + inf.w, we), gx, gy, gz);
            }
            __syncthreads();
        }
        // the force: the reactive entries' sum plus the others' (the order of
        // the resident step, so both paths give the same bits)
        fx = add_rn(fx, gx);
        fy = add_rn(fy, gy);
        fz = add_rn(fz, gz);
        // harmonic bonds (vitrimer chains): F_i = k (r - r0) (x_j - x_i) / r, half
        // of the energy and virial to each end (added to the two-body terms)
        if (BONDS && d.has_bonds && t < P) {  // BONDS: some system of the launch has bonds
            const P4 pi = SM::pos()[t];
            const int tag = pos_bits(pi) >> kTypeBits;
            for (int b = 0; b < kMaxBonds; b++) {
                const int pt = d.bond_tag[tag * kMaxBonds + b];
                if (pt < 0) break;
                const P4 pj = pos[d.slot_of_tag[pt]];
                Real dx, dy, dz;
                const Real r = sqrt(dist2_listed(pi, pj, d, dx, dy, dz));
                const Real dr = r - d.bond_r0;
                const Real g = d.bond_k * dr / r;
                fx += g * dx;
                fy += g * dy;
                fz += g * dz;
                if (!TH) continue;
                acc.q[Q_U2] += Real(0.25) * d.bond_k * dr * dr;
                const Real hf = Real(-0.5) * g;
                acc.q[Q_W0 + 0] += hf * dx * dx;
                acc.q[Q_W0 + 1] += hf * dy * dy;
                acc.q[Q_W0 + 2] += hf * dz * dz;
                acc.q[Q_W0 + 3] += hf * dx * dy;
                acc.q[Q_W0 + 4] += hf * dx * dz;
                acc.q[Q_W0 + 5] += hf * dy * dz;
            }
        }
        // FP32: park the thermo accumulators in the (now free) wave buffer while
        // the integrator runs, so they do not hold registers at its peak
        constexpr bool kPark = TH && sizeof(Real) == 4;
        if (kPark)
#pragma unroll
            for (int q = 0; q < kNQA; q++) SM::w()[q * blockDim.x + t] = acc.q[q];
        Real kin = Real(0);
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
            st.v = SM::vel()[t];
            if (flags & F_OPENING)
                for (int c = 0; c < 3; c++) st.q[c] = SM::xq()[3 * t + c];
            dmax = fmaxf(dmax, integrate_one(d, a, pc, ac, i, fx, fy, fz, flags, step, st, pos_bits(SM::pos()[t]),
                                             kin, single ? &SM::pos()[t] : (P4*)nullptr));
        }
        if (kPark)
#pragma unroll
            for (int q = 0; q < kNQA; q++) acc.q[q] = SM::w()[q * blockDim.x + t];
        if (TH) acc.q[Q_K] += kin;
        __syncthreads();
        if (TH && !single) {
            // several sub-chunks: fold this one's terms into the block's FP64
            // running sums, so no thread accumulates more than one sub-chunk
            // (per-warp running sums without the block barriers, tried in FP64
            // and in double-float, measured slower)
            block_sums(acc.q, SM::w(), blk, (double*)nullptr);
#pragma unroll
            for (int q = 0; q < kNQA; q++) acc.q[q] = Real(0);
        }
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
    const typename Dev<Real>::P4 pi = d.pos[pc][i];
    PState<Real> st;
    load_pstate(d, ac, i, F_OPENING, st);
    Real unused = Real(0);
    return integrate_one(d, a, pc, ac, i, f.x, f.y, f.z, F_OPENING, step, st, pos_bits(pi), unused,
                         (typename Dev<Real>::P4*)nullptr);
}

// ---------------------------------------------------------------------------
// The persistent step kernel.  One cooperative launch advances a.nsteps time
// steps (or only rebuilds, or only brings the forces up to date), with two
// grid barriers per step and a rebuild whenever the accumulated displacement
// bound can let an unlisted pair come inside its cut-off.
//
// Block-wide state lives in shared memory at namespace scope (addressed
// directly, not through pointers), so that nothing but the phase at hand
// occupies registers: the kernel runs at the 80-register limit of a
// 768-thread block.

struct LoopState {
    unsigned long long bar_target;  // barrier generation target (thread 0)
    long long step;
    long long rebuilds;
    int state, pc, ac, need_rb, remaining, done, have_thermo, rc, ok;
    float disp;
    unsigned dmax_bits;  // the block's largest squared step displacement (float bits)
    int own_ok;          // shared positions and list ranges of the block's particles are current
    // resident mode (section below)
    int r_try;           // build the resident structures before the next step
    int r_valid;         // every block's resident structures are built and current
    int r_gathered;      // the next step's copies were issued after the last barrier
    int r_round;         // agreement round (selects ctl->rfail[round & 1])
    int r_fail;          // this block's structures do not fit
    int r_np, r_nh, r_nhr;  // own particles, halo particles, halo rows of S
    int r_steps;         // steps this launch took in the resident mode
    int tlog_left;       // steps up to and including the next logged one (0: no log)
    int tlog_slot;       // ring slot of the next thermo-log record
    int tlog_k;          // records this launch wrote
};

static __shared__ __align__(16) unsigned char s_tab_raw[kMaxTypes * kMaxTypes * sizeof(PairP<double>)];
static __shared__ double s_red[32];
static __shared__ double s_blk[kNQ];  // the block's FP64 running thermo sums of the current pass
static __shared__ int s_int[64];
static __shared__ LoopState s_ls;

template <typename Real>
__device__ __forceinline__ const PairP<Real>* stab() { return (const PairP<Real>*)s_tab_raw; }

__device__ __forceinline__ bool grid_barrier(Ctl* ctl, long long timeout_ns, int where,
                                             unsigned* pub_dst = nullptr)
{
    BarState bs;
    bs.target = s_ls.bar_target;
    bar_arrive(ctl, bs, pub_dst, &s_ls.dmax_bits);
    if (threadIdx.x == 0) s_ls.bar_target = bs.target;
    return bar_wait(ctl, bs, timeout_ns, where, &s_ls.ok);
}

// 0: ok; 1: the list overflowed its capacity; 2: a wait timed out.
template <typename Real>
__device__ SWP_COLD int run_rebuild(const Dev<Real>& d, const RunArgs& a)
{
    Ctl* ctl = d.ctl;
    const int gt = g_rank() * blockDim.x + threadIdx.x, gn = g_size() * blockDim.x;
    if (threadIdx.x == 0 && g_rank() == 0) {
        ctl->max_row = 0;
        ctl->overflow = 0;
    }
    const int pc0 = s_ls.pc, ac0 = s_ls.ac;
    ph_bin(d, pc0, gt, gn);  // cell counts start at zero (see ph_chunk_scan)
    if (!grid_barrier(ctl, a.timeout_ns, 1)) return 2;
    ph_chunk_sums(d, s_int);
    if (!grid_barrier(ctl, a.timeout_ns, 2)) return 2;
    ph_chunk_scan(d, s_int);
    if (!grid_barrier(ctl, a.timeout_ns, 3)) return 2;
    ph_scatter(d, gt, gn);
    if (!grid_barrier(ctl, a.timeout_ns, 4)) return 2;
    ph_cell_sort(d, gt, gn);
    if (!grid_barrier(ctl, a.timeout_ns, 5)) return 2;
    ph_gather(d, pc0, ac0, gt, gn);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ls.pc = pc0 ^ 1;
        s_ls.ac = ac0 ^ 1;
    }
    if (!grid_barrier(ctl, a.timeout_ns, 6)) return 2;
    int ovf = 0;
    const int need = ph_build_cells<Real>(d, stab<Real>(), pc0 ^ 1, (int2*)Stage<Real>::w(), s_int, &ovf);
    if (threadIdx.x == 0) {
        atomicMax(&ctl->max_row, need);
        if (ovf) atomicOr(&ctl->overflow, 1);
    }
    if (!grid_barrier(ctl, a.timeout_ns, 7)) return 2;
    const int any_ovf = ld_relaxed(&ctl->overflow);
    if (threadIdx.x == 0) {
        s_ls.rebuilds++;
        s_ls.disp = 0.0f;
        s_ls.own_ok = 0;  // the particles were reordered
    }
    __syncthreads();
    if (any_ovf) {
        if (gt == 0) atomicOr(&ctl->status, kStatusOverflow);
        return 1;
    }
    return 0;
}

// One sub-chunk per block: the block's particles fit one shared staging.
template <typename Real>
__device__ __forceinline__ bool single_chunk(const Dev<Real>& d)
{
    return (d.n + g_size() - 1) / g_size() <= (int)blockDim.x;
}

template <typename Real, bool UNI>
__device__ __forceinline__ void run_s_pass(const Dev<Real>& d, const RunArgs& a)
{
    const bool single = single_chunk(d);
    s_pass_block<Real, UNI>(d, stab<Real>(), s_ls.pc, uni_params(a, Real(0))[0], single && s_ls.own_ok);
    if (threadIdx.x == 0) s_ls.own_ok = single;  // every thread read it before the pass's barriers
}

// Folds a thread's squared displacement into the block's shared maximum (one
// shared atomic per warp); the barrier arrival publishes it.
__device__ __forceinline__ void warp_max_disp(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0f) atomicMax(&s_ls.dmax_bits, __float_as_uint(v));
}

template <typename Real, bool UNI, bool BONDS, bool TH>
__device__ __forceinline__ void run_f_pass(const Dev<Real>& d, const RunArgs& a, int flags, long long stp,
                                           Acc<Real>& acc)
{
#pragma unroll
    for (int q = 0; q < kNQA; q++) acc.q[q] = Real(0);
    const float dmax = f_pass_block<Real, UNI, BONDS, TH>(d, stab<Real>(), a, s_ls.pc, s_ls.ac, flags, stp, acc,
                                                      uni_params(a, Real(0))[0], uni_params(a, Real(0))[1], s_blk);
    if (flags & F_OPENING) warp_max_disp(dmax);
}

template <typename Real>
__device__ void run_open_pass(const Dev<Real>& d, const RunArgs& a, long long stp)
{
    float dmax = 0.0f;
    const int pc = s_ls.pc, ac = s_ls.ac;
    for (int i = g_rank() * blockDim.x + threadIdx.x; i < d.n; i += g_size() * blockDim.x)
        dmax = fmaxf(dmax, open_from_stored(d, a, pc, ac, i, stp));
    warp_max_disp(dmax);
}

// Deterministic reduction of the block partials of the sampled step: block q
// sums quantity q over all blocks in a fixed order.
template <typename Real>
__device__ void run_reduce_thermo(const Dev<Real>& d)
{
    const int G = g_size(), nwp = (G + 31) / 32;
    const int lw = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = g_rank(); q < kNQA; q += G) {  // block-uniform loop
        if (w < nwp) {
            const int b = threadIdx.x;
            double v = b < G ? d.partials[(size_t)b * kNQ + q] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lw == 0) s_red[w] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < nwp; k++) t += s_red[k];
            d.ctl->thermo[q] = t;
        }
        __syncthreads();
    }
}

// The same reduction for a group of fewer than kNQA blocks (batched runs):
// rank 0 alone, warp q summing quantity q over the group's blocks in order.
template <typename Real>
__device__ __forceinline__ void reduce_small(const Dev<Real>& d)
{
    if (g_rank() != 0) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    for (int q = w; q < kNQA; q += nw) {
        double v = lane < g_size() ? d.partials[(size_t)lane * kNQ + q] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) d.ctl->thermo[q] = v;
    }
}

// Writes the block's partials of a sampled step's thermo terms (energies,
// virial, bond count, kinetic energy) from the threads' accumulators (or, for
// a resident step, from the per-warp sums s_wpart it left) to the launch's
// partials (last: the last step of the launch, whose values the launch
// reports; reduced after the loop) and/or to a thermo-log record (log).
// Every call is followed by a grid barrier.  Steps that are neither the
// launch's last nor logged skip the thermo terms altogether.
template <typename Real>
__device__ __forceinline__ void thermo_partials(const Dev<Real>& d, const Acc<Real>& acc, Real* stage,
                                                bool folded, bool last, double* log)
{
    double* out = last ? d.partials + (size_t)g_rank() * kNQ : log;
    double* out2 = last ? log : nullptr;
    if (folded)
        block_sums_from_warps(s_blk, out, out2);
    else
        block_sums(acc.q, stage, s_blk, out, out2);
    if (last && threadIdx.x == 0) s_ls.have_thermo = 1;
}

__device__ __forceinline__ void add_disp(Ctl* ctl, long long stp)
{
    if (threadIdx.x == 0)
        s_ls.disp += sqrtf(__uint_as_float((unsigned)ld_relaxed((const int*)&ctl->dmax2[stp & 1])));
    __syncthreads();
}

#if SWP_HAS_RESIDENT
// ---------------------------------------------------------------------------
// Resident mode: one system, FP32, no bonds, every block's particles in one
// sub-chunk (up to blockDim x grid particles).
//
// After each list build every block copies into shared memory what its steps
// need: the snapshots of its own particles and of its halo -- every particle
// outside the block that is a list partner of an own particle, plus every
// reactive partner of those that are reactive partners of an own particle --
// the own rows, and the reactive rows of that first halo shell (each the
// owner's row, in the owner's order), all with partners as 16-bit local
// indices.  A step then copies the halo's new snapshots in once (one
// asynchronous 16-byte copy each), forms S for the own particles and for the reactive halo
// from shared memory (a halo row is its owner's row, evaluated in the same
// order with the same operations, so both blocks hold bit-identical S), and
// the pair forces and the integrator with no further global gather: one grid
// barrier per step instead of two, and no chains of dependent L2 round trips
// inside a step.  Forces and trajectories are bit-identical to the two-barrier
// path (same per-entry operations, same summation orders); only the thermo
// partials are grouped differently.

struct RStage {
    static constexpr int kL = 3072;    // local particles: own (at most blockDim), then halo
    static constexpr int kES = 16384;  // entries of the rows of S, warp-major (padded to each warp's longest)
    static constexpr int kEF = 12288;  // entries of the own rows (force pass), laid out the same way
    static constexpr int kHash = 4096; // open-addressing table of halo slots (while building)
    static constexpr int kRounds = (kL + kBlock - 1) / kBlock;  // rows of S per thread, at most
    static constexpr size_t O_LPOS = 0;                             // [kL] int4 snapshots (own, then halo)
    static constexpr size_t O_LS = O_LPOS + (size_t)kL * 16;        // [kL] float S
    static constexpr size_t O_HSLOT = O_LS + (size_t)kL * 4;        // [kL] int global slot of halo particle h
    static constexpr size_t O_SENT = O_HSLOT + (size_t)kL * 4;      // [kES] u16 local partners of the rows of S
    static constexpr size_t O_FENT = O_SENT + (size_t)kES * 2;      // [kEF] u16 local partners of the own rows
    static constexpr size_t O_SDESC = O_FENT + (size_t)kEF * 2;     // [kL] int2 row of S: (lane's first entry, centre | n << 16)
    static constexpr size_t O_FDESC = O_SDESC + (size_t)kL * 8;     // [kBlock] int4 by thread: (first entry of its
                                                                    // reactive row, of its other row, nr | nw << 16,
                                                                    // centre of each (16 bits each, 0xffff: none))
    static constexpr size_t O_FW = O_FDESC + (size_t)kBlock * 16;   // [3][kBlock] float other-row forces by centre
    // the own particles' state, by row position, kept here between list builds
    // (global memory is brought up to date by r_flush)
    static constexpr size_t O_VEL = O_FW + (size_t)kBlock * 12;     // [kBlock] float4 velocities
    static constexpr size_t O_XQ = O_VEL + (size_t)kBlock * 16;     // [3 kBlock] fixed-point positions
    static constexpr size_t O_IMG = O_XQ + (size_t)kBlock * 24;     // [3 kBlock] image counts
    static constexpr size_t kBytes = O_IMG + (size_t)kBlock * 12;
    // While building, the own-state area holds the hash table (keys, values),
    // the sort histogram and the warp-block lengths; O_SENT holds the
    // reactive first shell's table indices, O_LS the centres of the rows of S
    // by position.
    static constexpr size_t B_KEY = O_VEL, B_VAL = B_KEY + (size_t)kHash * 4, B_HIST = B_VAL + (size_t)kHash * 4,
                            B_WL = B_HIST + 256 * 4, B_END = B_WL + ((size_t)kRounds * 32 + 1) * 4;
    static_assert(B_END <= kBytes, "build scratch fits the own-state area");
    static_assert(kES <= 65536 && kEF <= 65536 && kL <= 65536, "16-bit local indices and offsets");
    static_assert(kBlock % 32 == 0 && kBlock / 32 <= 32, "whole warps, at most 32");
    static_assert(kBlock >= 256 && kEF >= kBlock / 32 * 256, "force-row sort scratch (r_rank1_desc) in O_FENT");

    static __device__ __forceinline__ int4* lpos() { return (int4*)(g_dyn + O_LPOS); }
    static __device__ __forceinline__ float* lS() { return (float*)(g_dyn + O_LS); }
    static __device__ __forceinline__ int* hslot() { return (int*)(g_dyn + O_HSLOT); }
    static __device__ __forceinline__ unsigned short* sent() { return (unsigned short*)(g_dyn + O_SENT); }
    static __device__ __forceinline__ unsigned short* fent() { return (unsigned short*)(g_dyn + O_FENT); }
    static __device__ __forceinline__ int2* sdesc() { return (int2*)(g_dyn + O_SDESC); }
    static __device__ __forceinline__ int4* fdesc() { return (int4*)(g_dyn + O_FDESC); }
    static __device__ __forceinline__ float* fw() { return (float*)(g_dyn + O_FW); }
    static __device__ __forceinline__ float4* vel() { return (float4*)(g_dyn + O_VEL); }
    static __device__ __forceinline__ long long* xq() { return (long long*)(g_dyn + O_XQ); }
    static __device__ __forceinline__ int* img() { return (int*)(g_dyn + O_IMG); }
};
static_assert(RStage::kBytes <= Stage<float>::kBytes + 32768, "the resident layout fits the kernel's shared memory");

__device__ __forceinline__ void cp_async_cg16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ unsigned r_hash(int q) { return ((unsigned)q * 2654435761u) >> 20; }

// Inserts slot q into the table (if absent); its index, or -1 when full.
__device__ __forceinline__ int r_insert(int* key, int q)
{
    unsigned h = r_hash(q) & (RStage::kHash - 1);
    for (int probe = 0; probe < RStage::kHash; probe++) {
        const int old = atomicCAS(&key[h], -1, q);
        if (old == -1 || old == q) return (int)h;
        h = (h + 1) & (RStage::kHash - 1);
    }
    return -1;
}

__device__ __forceinline__ int r_find(const int* key, int q)
{
    unsigned h = r_hash(q) & (RStage::kHash - 1);
    for (int probe = 0; probe < RStage::kHash; probe++) {
        const int k = key[h];
        if (k == q) return (int)h;
        if (k == -1) return -1;
        h = (h + 1) & (RStage::kHash - 1);
    }
    return -1;
}

// Local index of global slot q: own particles first (q - b0), then the halo
// (P + compact rank, kept in val >> 1).
__device__ __forceinline__ int r_lid(const int* key, const int* val, int q, int b0, int b1, int P, int& fail)
{
    if (q >= b0 && q < b1) return q - b0;
    const int h = r_find(key, q);
    if (h < 0) {
        fail = 1;
        return 0;
    }
    return P + (val[h] >> 1);
}

// Counting sort, largest key first, of up to R items per thread (keys in
// [0, 255], -1: no item); pos[r] gets item r's rank.  Equal keys keep the
// order (thread, then round), so the result is the same on every run.
template <int R>
__device__ void r_sort_desc(const int (&key)[R], int (&pos)[R], int* hist)
{
    const int t = threadIdx.x, B = blockDim.x;
    for (int h = t; h < 256; h += B) hist[h] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++)
        if (key[r] >= 0) atomicAdd(&hist[key[r]], 1);
    __syncthreads();
    int base = 0;
    for (int c = 255; c >= 0; c--) {
        if (hist[c] == 0) continue;  // the same in every thread
        int cl = 0;
#pragma unroll
        for (int r = 0; r < R; r++) cl += key[r] == c;
        int tot;
        int off = block_excl_scan(cl, s_int, &tot);
#pragma unroll
        for (int r = 0; r < R; r++)
            if (key[r] == c) pos[r] = base + off++;
        base += tot;
    }
}

// Stable counting sort, largest key first, of one item per thread (key in
// [0, 255], -1: no item): returns the item's rank.  Equal keys keep the thread
// order.  wh: scratch of blockDim / 32 x 256 u16 counts; hist: 256 ints;
// blockDim >= 256.
static __device__ int r_rank1_desc(int key, unsigned short* wh, int* hist)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, NW = blockDim.x >> 5;
    __syncthreads();  // a previous call's readers are done with wh and hist
    for (int k = t; k < NW * 256; k += blockDim.x) wh[k] = 0;
    __syncthreads();
    // the warp's lanes with this key, and how many come before this lane
    const unsigned m = __match_any_sync(0xffffffffu, key);
    const int before = __popc(m & ((1u << lane) - 1u));
    if (key >= 0 && before == 0) wh[warp * 256 + key] = (unsigned short)__popc(m);
    __syncthreads();
    // per key: the counts of the warps before each warp, and the key's total
    if (t < 256) {
        int run = 0;
        for (int w = 0; w < NW; w++) {
            const int c = wh[w * 256 + t];
            wh[w * 256 + t] = (unsigned short)run;
            run += c;
        }
        hist[t] = run;
    }
    __syncthreads();
    // keys in descending order: the first rank of key b is the count above it
    const int b = 255 - t;
    int tot;
    const int ex = block_excl_scan(t < 256 ? hist[b] : 0, s_int, &tot);
    if (t < 256) hist[b] = ex;  // every thread read hist before the scan's barriers
    __syncthreads();
    return key >= 0 ? hist[key] + wh[warp * 256 + key] + before : 0;
}

// Lays out warp blocks: rows at positions s (thread s % B, round s / B) with
// n[r] entries each (0: no row); every warp block of 32 rows takes 32 x its
// longest row, in order (round, warp).  Returns the total (entries), and in
// first[r] the entry of row r's lane (entry k of the row at first + 32 k).
template <int R>
__device__ int r_warp_layout(const int (&n)[R], int (&first)[R], int* wl)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int L = __reduce_max_sync(0xffffffffu, n[r]);
        if (lane == 0) wl[r * nw + warp] = L;
    }
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int b = 0; b < R * nw; b++) {
            const int L = wl[b];
            wl[b] = acc;
            acc += 32 * L;
        }
        wl[R * nw] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++) first[r] = wl[r * nw + warp] + lane;
    const int total = wl[R * nw];
    __syncthreads();
    return total;
}

// Builds the block's resident structures from the global list and the
// snapshots pos[pc].  Returns 1 when they fit (the same answer in every
// thread of the block); 0 leaves nothing the step relies on.
static __device__ int r_localize(const Dev<float>& d, int pc, int ac)
{
    typedef RStage RS;
    constexpr int RR = RS::kRounds;
    int4* lpos = RS::lpos();
    int* key = (int*)(g_dyn + RS::B_KEY);
    int* val = (int*)(g_dyn + RS::B_VAL);  // bit 0: reactive partner of an own particle; then the rank << 1
    int* hist = (int*)(g_dyn + RS::B_HIST);
    int* wl = (int*)(g_dyn + RS::B_WL);
    int* hr = (int*)RS::sent();   // table index of the k-th reactive first-shell particle
    int* cen = (int*)RS::lS();    // centre (local index) of the row at each position
    const int t = threadIdx.x, B = blockDim.x;
    const int PER = (RS::kHash + B - 1) / B;
    int b0, b1;
    block_range(d, b0, b1);
    const int P = b1 - b0;
    if (B != kBlock || P > B) return 0;
    for (int h = t; h < RS::kHash; h += B) {
        key[h] = -1;
        val[h] = 0;
    }
    __syncthreads();
    int fail = 0;
    int e_beg = 0, e_rend = 0, e_end = 0;
    if (P > 0) {
        const int4 f0 = d.pinfo[b0], f1 = d.pinfo[b1 - 1];
        e_beg = f0.x;
        e_rend = f1.x + f1.y;
        e_end = f1.z + f1.w;
    }
    // 1. first shell: the partners of the own rows outside the block
    for (int e = e_beg + t; e < e_end; e += B) {
        const int q = d.ent_j[e];
        if (q < b0 || q >= b1) {
            const int h = r_insert(key, q);
            if (h < 0) fail = 1;
            else if (e < e_rend) atomicOr(&val[h], 1);
        }
    }
    if (__syncthreads_or(fail)) return 0;
    // 2. its reactive part (their S is formed here too), in table order
    const int h0 = min(t * PER, RS::kHash), h1 = min(h0 + PER, RS::kHash);
    int c = 0;
    for (int h = h0; h < h1; h++) c += val[h] & 1;
    int Hr;
    int off = block_excl_scan(c, s_int, &Hr);
    if (P + Hr > RS::kL) return 0;  // Hr is the same in every thread
    for (int h = h0; h < h1; h++)
        if (val[h] & 1) hr[off++] = h;
    __syncthreads();
    // 3. second shell: the reactive partners of the reactive first shell
    for (int k = t; k < Hr; k += B) {
        const int4 fi = d.pinfo[key[hr[k]]];
        for (int e = fi.x; e < fi.x + fi.y; e++) {
            const int q = d.ent_j[e];
            if ((q < b0 || q >= b1) && r_insert(key, q) < 0) fail = 1;
        }
    }
    if (__syncthreads_or(fail)) return 0;
    // 4. compact the table: halo particle of rank r has local index P + r
    c = 0;
    for (int h = h0; h < h1; h++) c += key[h] != -1;
    int H;
    off = block_excl_scan(c, s_int, &H);
    if (P + H > RS::kL) return 0;
    for (int h = h0; h < h1; h++) {
        if (key[h] != -1) {
            RS::hslot()[off] = key[h];
            val[h] = (val[h] & 1) | (off << 1);
            off++;
        }
    }
    __syncthreads();
    // 5. rows of S (the own rows and the reactive first shell's), longest
    // first, dealt out over the threads as a snake: rank s goes to round
    // s / B, to thread s % B in even rounds and B - 1 - s % B in odd ones, so
    // that a thread's second row is short when its first is long.  The force
    // pass runs two loops per thread, over a reactive row and over another
    // particle's other (purely two-body) row: reactive rows longest first
    // from warp 0, other rows longest first from the last warp, so that the
    // rows of a warp are alike in each loop and the warps' totals even out.
    const int NS = P + Hr;
    const int rounds = (NS + B - 1) / B;
    int4 inf = make_int4(0, 0, 0, 0);
    if (t < P) inf = d.pinfo[b0 + t];
    if (inf.y > 255 || inf.w > 255) fail = 1;
    int skey[RR + 1], spos[RR + 1], hrow[RR], hcnt[RR];
    skey[0] = t < P ? min(inf.y, 255) : -1;
    spos[0] = 0;
#pragma unroll
    for (int r = 0; r < RR; r++) {
        const int k = t + r * B;
        skey[r + 1] = -1;
        spos[r + 1] = 0;
        hrow[r] = hcnt[r] = 0;
        if (k < Hr) {
            const int4 fi = d.pinfo[key[hr[k]]];
            hrow[r] = fi.x;
            hcnt[r] = fi.y;
            if (fi.y > 255) fail = 1;
            skey[r + 1] = min(fi.y, 255);
        }
    }
    r_sort_desc<RR + 1>(skey, spos, hist);
    const int W32 = (P + 31) & ~31;
    const int rpos = r_rank1_desc(t < P ? inf.y : -1, RS::fent(), hist);
    const int wrank = r_rank1_desc(t < P ? inf.w : -1, RS::fent(), hist);
    const int wpos = W32 - 32 - (wrank & ~31) + (wrank & 31);  // rank chunk c -> warp W32/32 - 1 - c
    for (int q = t; q < rounds * B; q += B) RS::sdesc()[q] = make_int2(0, -1);  // no row here
    if (t < W32) RS::fdesc()[t] = make_int4(0, 0, 0, -1);  // no rows; centres 0xffff
    __syncthreads();
    // what each position needs: the centre and the row (start, count)
#pragma unroll
    for (int r = 0; r <= RR; r++) {
        if (skey[r] < 0) continue;
        const int sr = spos[r], g = sr / B, slot = sr - g * B;
        const int q = g * B + ((g & 1) ? B - 1 - slot : slot);
        if (r == 0) {
            cen[q] = t;
            RS::sdesc()[q] = make_int2(inf.x, inf.y);
        } else {
            const int k = t + (r - 1) * B;
            cen[q] = P + (val[hr[k]] >> 1);
            RS::sdesc()[q] = make_int2(hrow[r - 1], hcnt[r - 1]);
        }
    }
    if (t < P) {
        // 16-bit fields: (z, w) = (nr, nw, reactive centre, other centre)
        int4* fr = &RS::fdesc()[rpos];
        int4* fo = &RS::fdesc()[wpos];
        fr->x = inf.x;
        fo->y = inf.z;
        ((unsigned short*)&fr->z)[0] = (unsigned short)inf.y;
        ((unsigned short*)&fo->z)[1] = (unsigned short)inf.w;
        ((unsigned short*)&fr->w)[0] = (unsigned short)t;
        ((unsigned short*)&fo->w)[1] = (unsigned short)t;
    }
    if (__syncthreads_or(fail)) return 0;
    // 6. warp-major layouts: the rows of S; the own rows' reactive parts, then
    // their other parts
    int n[RR], first[RR];
#pragma unroll
    for (int r = 0; r < RR; r++) {
        const int q = t + r * B;
        n[r] = r < rounds ? max(RS::sdesc()[q].y, 0) : 0;
    }
    const int ES = r_warp_layout<RR>(n, first, wl);
    const int4 fd = t < W32 ? RS::fdesc()[t] : make_int4(0, 0, 0, -1);
    int nrc[1] = {fd.z & 0xffff}, nwc[1] = {(int)((unsigned)fd.z >> 16)}, rfirst[1], wfirst[1];
    const int ER = r_warp_layout<1>(nrc, rfirst, wl);
    const int EW = r_warp_layout<1>(nwc, wfirst, wl);
    if (ES > RS::kES || ER + EW > RS::kEF) return 0;  // the same in every thread
    // 7. the rows, partners as local indices
#pragma unroll
    for (int r = 0; r < RR; r++) {
        const int q = t + r * B;
        if (r < rounds) {
            const int2 src = RS::sdesc()[q];
            if (src.y >= 0) {
                const int lid = cen[q];
                for (int m = 0; m < src.y; m++)
                    RS::sent()[first[r] + 32 * m] =
                        (unsigned short)r_lid(key, val, d.ent_j[src.x + m], b0, b1, P, fail);
                RS::sdesc()[q] = make_int2(first[r], lid | (src.y << 16));
            }
        }
    }
    if (t < W32) {
        unsigned short* fe = RS::fent();
        for (int m = 0; m < nrc[0]; m++)
            fe[rfirst[0] + 32 * m] = (unsigned short)r_lid(key, val, d.ent_j[fd.x + m], b0, b1, P, fail);
        for (int m = 0; m < nwc[0]; m++)
            fe[ER + wfirst[0] + 32 * m] = (unsigned short)r_lid(key, val, d.ent_j[fd.y + m], b0, b1, P, fail);
        RS::fdesc()[t] = make_int4(rfirst[0], ER + wfirst[0], fd.z, fd.w);
    }
    if (t < P) lpos[t] = d.pos[pc][b0 + t];  // own snapshots by local index
    if (t == 0) {
        s_ls.r_np = P;
        s_ls.r_nh = H;
        s_ls.r_nhr = Hr;
    }
    const int ok = __syncthreads_or(fail) ? 0 : 1;
    // 8. the own particles' state by reactive-row position (over the table, now unused)
    if (ok && t < P) {
        const int i = b0 + (RS::fdesc()[t].w & 0xffff), n = d.n;
        RS::vel()[t] = d.vel[ac][i];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            RS::xq()[3 * t + c] = d.xq[ac][c * n + i];
            RS::img()[3 * t + c] = d.img[ac][c * n + i];
        }
    }
    __syncthreads();
    return ok;
}

// Writes the own particles' state back to the global arrays (set ac): before
// a list build reorders them, and when the run ends.
__device__ __forceinline__ void r_flush(const Dev<float>& d, int ac)
{
    typedef RStage RS;
    const int t = threadIdx.x, n = d.n;
    if (t < s_ls.r_np) {
        int b0, b1;
        block_range(d, b0, b1);
        const int i = b0 + (RS::fdesc()[t].w & 0xffff);
        d.vel[ac][i] = RS::vel()[t];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            d.xq[ac][c * n + i] = RS::xq()[3 * t + c];
            d.img[ac][c * n + i] = RS::img()[3 * t + c];
        }
    }
}

// Issues a step's copies of the halo's snapshots pos[pc] (through L2 only:
// other blocks wrote them).
__device__ __forceinline__ void r_gather(const Dev<float>& d, int pc)
{
    typedef RStage RS;
    const int t = threadIdx.x, B = blockDim.x, P = s_ls.r_np, H = s_ls.r_nh;
    int4* lpos = RS::lpos();
    const int* hslot = RS::hslot();
    const int4* pos = d.pos[pc];
    for (int h = t; h < H; h += B) cp_async_cg16(&lpos[P + h], &pos[hslot[h]]);
    cp_async_commit();
}

// S of one row (entries e[0], e[32], ...) with the two-barrier path's order of
// additions (groups of four, then one by one).
template <bool UNI>
__device__ __forceinline__ float r_row_s(const Dev<float>& d, const PairP<float>* tab, const PairP<float>& ps,
                                         const int4* lpos, const unsigned short* e, int cnt, const int4& pi)
{
    float s = 0.0f;
    int k = 0;
    for (; k + 4 <= cnt; k += 4) {
        const float w0 = s_term<float, UNI>(d, tab, ps, pi, lpos[e[32 * k]]);
        const float w1 = s_term<float, UNI>(d, tab, ps, pi, lpos[e[32 * (k + 1)]]);
        const float w2 = s_term<float, UNI>(d, tab, ps, pi, lpos[e[32 * (k + 2)]]);
        const float w3 = s_term<float, UNI>(d, tab, ps, pi, lpos[e[32 * (k + 3)]]);
        s += (w0 + w1) + (w2 + w3);
    }
    for (; k < cnt; k++) s += s_term<float, UNI>(d, tab, ps, pi, lpos[e[32 * k]]);
    return s;
}

// One resident step: S of the own particles and the reactive halo, the pair
// forces of the own rows (entry order: reactive, then the others), the
// integrator.  TH (the sampled step): the thermo terms are left summed per
// warp in s_wpart (thermo_partials completes the block sums).  Returns the
// thread's squared drift displacement.
template <bool UNI, bool TH>
__device__ float r_step(const Dev<float>& d, const RunArgs& a, int flags, long long step, Acc<float>& acc)
{
    typedef RStage RS;
    const int t = threadIdx.x, B = blockDim.x;
    const int P = s_ls.r_np, NQ = (P + s_ls.r_nhr + B - 1) / B * B;  // positions of the rows of S
    const int pc = s_ls.pc;
    int b0, b1;
    block_range(d, b0, b1);
    if (!s_ls.r_gathered) r_gather(d, pc);
    cp_async_wait_all();
    __syncthreads();
    const PairP<float>* tab = stab<float>();
    const PairP<float>& ps = a.uf[0];
    const PairP<float>& pw = a.uf[1];
    int4* lpos = RS::lpos();
    float* lS = RS::lS();
    for (int q = t; q < NQ; q += B) {
        const int2 dsc = RS::sdesc()[q];
        if (dsc.y < 0) continue;  // no row at this position
        const int lid = dsc.y & 0xffff;
        lS[lid] = r_row_s<UNI>(d, tab, ps, lpos, RS::sent() + dsc.x, (int)((unsigned)dsc.y >> 16), lpos[lid]);
    }
    __syncthreads();
    if (TH)
#pragma unroll
        for (int q = 0; q < kNQA; q++) acc.q[q] = 0.0f;
    float dmax = 0.0f, kin = 0.0f;
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    int4 pi = make_int4(0, 0, 0, 0);
    int lid = 0;
    float* fw = RS::fw();
    if (t < ((P + 31) & ~31)) {
        const int4 fd = RS::fdesc()[t];
        const int nr = fd.z & 0xffff, nw = (int)((unsigned)fd.z >> 16);
        const int cw = (int)((unsigned)fd.w >> 16);
        lid = fd.w & 0xffff;
        if (cw != 0xffff) {
            // the other (purely two-body) row of particle cw: its sum goes to
            // fw, for the thread that integrates cw
            const unsigned short* ew = RS::fent() + fd.y;
            const int4 pc_ = lpos[cw];
            float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll 2
            for (int k = 0; k < nw; k++) {
                const int j = ew[32 * k];
                float ex, ey, ez;
                entry_force<float, UNI, false, TH>(d, tab, pc_, lpos[j], 0.0f, 0.0f, pw, acc, ex, ey, ez);
                gx = __fadd_rn(gx, ex);
                gy = __fadd_rn(gy, ey);
                gz = __fadd_rn(gz, ez);
            }
            fw[cw] = gx;
            fw[kBlock + cw] = gy;
            fw[2 * kBlock + cw] = gz;
        }
        if (t < P) {
            // the reactive row of particle lid
            const unsigned short* er = RS::fent() + fd.x;
            pi = lpos[lid];
            const float Si = lS[lid];
#pragma unroll 2
            for (int k = 0; k < nr; k++) {
                const int j = er[32 * k];
                float ex, ey, ez;
                entry_force<float, UNI, true, TH>(d, tab, pi, lpos[j], Si, lS[j], ps, acc, ex, ey, ez);
                fx = __fadd_rn(fx, ex);
                fy = __fadd_rn(fy, ey);
                fz = __fadd_rn(fz, ez);
            }
        }
    }
    // the pair terms go to the warp partials now, so that the accumulators are
    // not live through the integrator (the kinetic term follows it)
    const bool rows = (t & ~31) < P;  // the warp holds rows (the same in all its lanes)
    if (TH) {
        if (rows) {
#pragma unroll
            for (int q = 0; q < kNQA; q++)
                if (q != Q_K) warp_part(acc.q[q], q);
        } else if ((t & 31) == 0) {
#pragma unroll
            for (int q = 0; q < kNQA; q++)
                if (q != Q_K) s_wpart[q][t >> 5] = 0.0f;
        }
    }
    __syncthreads();  // every row has read the old snapshots, and fw is complete
    if (t < P) {
        const int i = b0 + lid;
        // the force: the reactive row's sum plus the other row's
        fx = __fadd_rn(fx, fw[lid]);
        fy = __fadd_rn(fy, fw[kBlock + lid]);
        fz = __fadd_rn(fz, fw[2 * kBlock + lid]);
        if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(&d.ctl->status, kStatusNonfinite);
        if (flags & F_STORE) d.force[i] = make_float4(fx, fy, fz, 0.0f);
        float4 v = RS::vel()[t];
        long long q[3];
        int w[3];
#pragma unroll
        for (int c = 0; c < 3; c++) q[c] = RS::xq()[3 * t + c];
        int4 np = make_int4(0, 0, 0, 0);
        dmax = advance_particle(d, a, fx, fy, fz, flags, step, pi.w, v, q, w, kin, np);
        if (flags & F_OPENING) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                RS::xq()[3 * t + c] = q[c];
                RS::img()[3 * t + c] += w[c];
            }
            d.pos[pc ^ 1][i] = np;  // the other blocks' halos read it
            lpos[lid] = np;
        }
        RS::vel()[t] = v;
    }
    if (TH) {
        if (rows)
            warp_part(kin, Q_K);
        else if ((t & 31) == 0)
            s_wpart[Q_K][t >> 5] = 0.0f;
    }
    if (t == 0) {
        s_ls.r_gathered = 0;
        s_ls.r_steps++;
        s_ls.own_ok = 0;
    }
    return dmax;
}

// Builds every block's resident structures and agrees on the mode: the step
// runs resident only if every block's structures fit.
static __device__ bool r_enter(const Dev<float>& d, const RunArgs& a)
{
    const int ok = r_localize(d, s_ls.pc, s_ls.ac);
    const int round = s_ls.r_round;
    if (threadIdx.x == 0 && !ok) atomicOr(&d.ctl->rfail[round & 1], 1);
    if (!grid_barrier(d.ctl, a.timeout_ns, 8)) return false;
    if (threadIdx.x == 0) {
        s_ls.r_valid = ld_relaxed(&d.ctl->rfail[round & 1]) == 0;
        s_ls.r_try = 0;  // tried again after the next list build
        s_ls.r_round = round + 1;
        s_ls.r_gathered = 0;
        s_ls.own_ok = 0;  // the build overwrote the two-barrier path's staging
        // the next round's word: every block reads this round's word before it
        // arrives at the next barrier, and the next round comes after it
        if (g_rank() == 0) d.ctl->rfail[(round + 1) & 1] = 0;
    }
    __syncthreads();
    return true;
}

#endif  // SWP_HAS_RESIDENT

// One system advanced by the group of blocks this block belongs to (g_rank /
// g_size set by the caller).  Returns false when a wait timed out (the status
// word says so).
template <typename Real, bool UNI, bool BONDS>
__device__ __forceinline__ bool run_system(const Dev<Real>& d, const RunArgs& a)
{
    // the resident mode exists for one FP32 system without bonds
    constexpr bool kRes = SWP_HAS_RESIDENT && sizeof(Real) == 4 && !BONDS;
    Ctl* ctl = d.ctl;
    PairP<Real>* tab = (PairP<Real>*)s_tab_raw;
    const int ntt = d.ntypes * d.ntypes;
    for (int t = threadIdx.x; t < ntt; t += blockDim.x) tab[t] = d.table[t];
    if (threadIdx.x < kNQ) s_blk[threadIdx.x] = 0.0;
    if (threadIdx.x == 0) {
        s_withhold = a.withhold && g_rank() == 0;
        s_ls.bar_target = 0;
        s_ls.step = ctl->step;
        s_ls.rebuilds = 0;
        s_ls.state = ctl->state;
        s_ls.pc = ctl->pos_cur;
        s_ls.ac = ctl->arr_cur;
        // the list's block partition depends on the grid: rebuild if it changed
        s_ls.need_rb = ctl->need_rebuild | a.force_rebuild | (ctl->list_grid != g_size()) |
                       (ctl->list_chunk != (int)blockDim.x);
        s_ls.remaining = a.nsteps;
        s_ls.done = 0;
        s_ls.have_thermo = 0;
        s_ls.rc = 0;
        s_ls.disp = (float)ctl->disp;
        s_ls.dmax_bits = 0u;
        s_ls.own_ok = 0;
        s_ls.r_try = (kRes && a.resident && single_chunk(d)) ? 1 : 0;
        s_ls.r_valid = 0;
        s_ls.r_gathered = 0;
        s_ls.r_round = 0;
        s_ls.r_fail = 0;
        s_ls.r_np = s_ls.r_nh = s_ls.r_nhr = 0;
        s_ls.r_steps = 0;
        s_ls.tlog_left = 0;
        s_ls.tlog_slot = 0;
        s_ls.tlog_k = 0;
        if (a.tlog_every > 0 && d.tlog) {
            s_ls.tlog_left = a.tlog_every - (int)(s_ls.step % a.tlog_every);
            s_ls.tlog_slot = (int)(ctl->tlog_n % d.tlog_cap);
        }
        // both agreement words start clear: every round comes after a barrier
        if (kRes && g_rank() == 0) {
            ctl->rfail[0] = 0;
            ctl->rfail[1] = 0;
        }
    }
    __syncthreads();
    const float skin_eff = (float)a.skin_eff;

    if (a.build_only) {
        const int rc = run_rebuild(d, a);
        if (rc == 2) return false;
        if (threadIdx.x == 0) {
            s_ls.need_rb = rc;
            s_ls.rc = rc;
        }
        __syncthreads();
    } else {
        if (s_ls.state == 1) {
            if (s_ls.need_rb || 2.0f * s_ls.disp > skin_eff) {
                const int rc = run_rebuild(d, a);
                if (rc == 2) return false;
                if (threadIdx.x == 0) {
                    s_ls.need_rb = rc;
                    s_ls.rc = rc;
                }
                __syncthreads();
            }
            if (s_ls.rc == 0) {
                run_s_pass<Real, UNI>(d, a);
                if (!grid_barrier(ctl, a.timeout_ns, 10)) return false;
                Acc<Real> acc;
                run_f_pass<Real, UNI, BONDS, true>(d, a, F_STORE, s_ls.step, acc);
                if (threadIdx.x == 0) s_ls.state = 0;  // read again only after the barrier
                thermo_partials(d, acc, Stage<Real>::w(), false, true, (double*)nullptr);
                if (!grid_barrier(ctl, a.timeout_ns, 11)) return false;
            }
        }
        if (s_ls.rc == 0 && s_ls.remaining > 0 && s_ls.state == 0) {
            const long long stp = s_ls.step;
            if (threadIdx.x == 0 && g_rank() == 0) ctl->dmax2[stp & 1] = 0u;
            if (!grid_barrier(ctl, a.timeout_ns, 12)) return false;
            run_open_pass(d, a, stp);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_ls.pc ^= 1;
                s_ls.state = 2;
                s_ls.own_ok = 0;  // new positions in global memory only
            }
            if (!grid_barrier(ctl, a.timeout_ns, 13, &ctl->dmax2[stp & 1])) return false;
            add_disp(ctl, stp);
        }
        [[maybe_unused]] unsigned dm_pending = 0u;  // thread 0: the displacement maximum read after a resident barrier
        while (s_ls.rc == 0 && s_ls.state == 2) {
            const long long stp = s_ls.step;
            if (threadIdx.x == 0 && g_rank() == 0) ctl->dmax2[(stp + 1) & 1] = 0u;
#if SWP_HAS_RESIDENT
            if constexpr (kRes) {
                if (s_ls.r_gathered) {
                    // the halo copies and the displacement read issued after the
                    // last barrier were in flight together until here
                    cp_async_wait_all();
                    if (threadIdx.x == 0) s_ls.disp += sqrtf(__uint_as_float(dm_pending));
                    __syncthreads();
                }
            }
#endif
            if (s_ls.need_rb || 2.0f * s_ls.disp > skin_eff) {
                // a resident gather issued for this step lands in memory the rebuild reuses
                cp_async_wait_all();
#if SWP_HAS_RESIDENT
                if constexpr (kRes)
                    if (s_ls.r_valid) r_flush(d, s_ls.ac);  // the build reorders the global state
#endif
                const int rc = run_rebuild(d, a);
                if (rc == 2) return false;
                if (threadIdx.x == 0) {
                    s_ls.need_rb = rc;
                    s_ls.rc = rc;
                    s_ls.r_valid = 0;
                    s_ls.r_gathered = 0;
                    s_ls.r_try = (kRes && a.resident && single_chunk(d)) ? 1 : 0;
                }
                __syncthreads();
                if (rc) break;
            }
            const bool more = s_ls.remaining > 1;
            // the thermo terms are summed on the launch's last step (the one a
            // launch reports) and on the logged steps only
            const bool logged = s_ls.tlog_left == 1;
            const bool th = !more || logged;
            const int flags = F_CLOSING | (more ? F_OPENING : F_STORE);
            Acc<Real> acc;
            bool resident = false;
#if SWP_HAS_RESIDENT
            if constexpr (kRes) {
                if (s_ls.r_try)
                    if (!r_enter(d, a)) return false;
                if (s_ls.r_valid) {
                    const float dmax = th ? r_step<UNI, true>(d, a, flags, stp + 1, acc)
                                          : r_step<UNI, false>(d, a, flags, stp + 1, acc);
                    if (more) warp_max_disp(dmax);
                    resident = true;
                }
            }
#endif
            if (!resident) {
                run_s_pass<Real, UNI>(d, a);
                if (!grid_barrier(ctl, a.timeout_ns, 20)) return false;
                if (th)
                    run_f_pass<Real, UNI, BONDS, true>(d, a, flags, stp + 1, acc);
                else
                    run_f_pass<Real, UNI, BONDS, false>(d, a, flags, stp + 1, acc);
            }
            if (threadIdx.x == 0) {  // every thread read `remaining` before the pass's barriers
                s_ls.step = stp + 1;
                s_ls.remaining--;
                s_ls.done++;
                if (s_ls.tlog_left > 0) s_ls.tlog_left = logged ? a.tlog_every : s_ls.tlog_left - 1;
            }
            double* lg = logged ? d.tlog + ((size_t)s_ls.tlog_slot * a.max_blocks + g_rank()) * kNQ : nullptr;
            if (logged && threadIdx.x == 0 && g_rank() == 0) {
                d.tlog_step[2 * s_ls.tlog_slot] = stp + 1;
                d.tlog_step[2 * s_ls.tlog_slot + 1] = g_size();
            }
            // a logged resident step that is not the launch's last sums its
            // warps' thermo terms while it waits at the barrier (the record is
            // read after the launch); the launch's last step writes the
            // partials the launch reduces, before its arrival
            const bool late = resident && more;
            if (th && !late) thermo_partials(d, acc, Stage<Real>::w(), resident, !more, lg);
            unsigned* pub = more ? &ctl->dmax2[(stp + 1) & 1] : nullptr;
            {
                BarState bs;
                bs.target = s_ls.bar_target;
                bar_arrive(ctl, bs, pub, &s_ls.dmax_bits);
                if (th && late) warp_sums_to(s_blk, lg, nullptr);  // bar_arrive ordered the s_wpart writes
                if (threadIdx.x == 0) s_ls.bar_target = bs.target;
                if (!bar_wait(ctl, bs, a.timeout_ns, 21, &s_ls.ok)) return false;
            }
            if (logged && threadIdx.x == 0) {  // every thread used the slot before the barrier
                s_ls.tlog_k++;
                s_ls.tlog_slot = s_ls.tlog_slot + 1 == d.tlog_cap ? 0 : s_ls.tlog_slot + 1;
            }
            if (more) {
                if (threadIdx.x == 0) s_ls.pc ^= 1;
                __syncthreads();
                bool gathered = false;
#if SWP_HAS_RESIDENT
                if constexpr (kRes) {
                    if (s_ls.r_valid) {
                        // the displacement read and the next step's copies
                        // overlap; the read is used after the copies land (top
                        // of the loop)
                        if (threadIdx.x == 0) dm_pending = (unsigned)ld_relaxed((const int*)pub);
                        r_gather(d, s_ls.pc);
                        if (threadIdx.x == 0) s_ls.r_gathered = 1;
                        __syncthreads();
                        gathered = true;
                    }
                }
#endif
                if (!gathered) add_disp(ctl, stp + 1);
            } else {
                if (threadIdx.x == 0) s_ls.state = 0;
                __syncthreads();
            }
        }
    }
    cp_async_wait_all();  // copies issued for a step that did not come
#if SWP_HAS_RESIDENT
    if constexpr (kRes)
        if (s_ls.r_valid) r_flush(d, s_ls.ac);
#endif
    if (s_ls.have_thermo) {
        // the partials were written before the arrival at the barrier that
        // followed their pass, which every block has passed
        if (kBatched && g_size() < kNQA)
            reduce_small(d);
        else
            run_reduce_thermo(d);
    }
    if (g_rank() == 0 && threadIdx.x == 0) {
        ctl->state = s_ls.state;
        ctl->pos_cur = s_ls.pc;
        ctl->arr_cur = s_ls.ac;
        ctl->step = s_ls.step;
        ctl->disp = s_ls.disp;
        ctl->n_rebuilds += s_ls.rebuilds;
        ctl->steps_done = s_ls.done;
        ctl->need_rebuild = s_ls.need_rb;
        ctl->resident_steps = s_ls.r_steps;
        ctl->tlog_n += s_ls.tlog_k;
        if (s_ls.rebuilds > 0) {
            ctl->list_grid = s_ls.rc == 0 ? g_size() : -1;
            ctl->list_chunk = blockDim.x;
        }
    }
    return true;
}

#if !SWP_BATCHED
template <typename Real, bool UNI, bool BONDS>
__global__ void __launch_bounds__(kThreads, 1) k_run(Dev<Real> d, RunArgs a)
{
    run_system<Real, UNI, BONDS>(d, a);
}
#else

// Batched launch: many independent systems in one cooperative launch.  Block
// b works through items[item_ofs[b] .. item_ofs[b + 1]), each (system, rank in
// the system's group, group size): a system either has a group of blocks to
// itself or runs on one block, which then advances its systems one after the
// other.  A block that belongs to a group of more than one block has no other
// item, so the group barriers only ever wait for blocks working on the same
// system.
template <typename Real, bool UNI, bool BONDS>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_batch(const Dev<Real>* devs, const RunArgs* args,
                                                     const int* item_ofs, const int4* items)
{
    __shared__ Dev<Real> s_dev;
    __shared__ RunArgs s_args;
    const int i0 = item_ofs[blockIdx.x], i1 = item_ofs[blockIdx.x + 1];
    for (int it = i0; it < i1; it++) {
        const int4 w = items[it];
        __syncthreads();  // the previous system is done with the shared copies
        const int* sd = (const int*)&devs[w.x];
        const int* sa = (const int*)&args[w.x];
        for (int k = threadIdx.x; k < (int)(sizeof(Dev<Real>) / 4); k += blockDim.x) ((int*)&s_dev)[k] = sd[k];
        for (int k = threadIdx.x; k < (int)(sizeof(RunArgs) / 4); k += blockDim.x) ((int*)&s_args)[k] = sa[k];
        if (threadIdx.x == 0) {
            s_grp[0] = w.y;
            s_grp[1] = w.z;
        }
        __syncthreads();
        if (!run_system<Real, UNI, BONDS>(s_dev, s_args)) {
            // a wait of this system ran out (latched in its status word): its
            // copies in flight land before the next system reuses the shared
            // buffers, and the block goes on with its other systems
            cp_async_wait_all();
            __syncthreads();
        }
    }
}
#endif  // SWP_BATCHED

#if SWP_HAS_RESIDENT
// ---------------------------------------------------------------------------
// Host-exchange kernels (user order <-> slot order).

template <typename Real>
__global__ void k_set_state(Dev<Real> d)
{
    typedef typename Dev<Real>::R4 R4;
    typedef typename Dev<Real>::P4 P4;
    const int n = d.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        long long qs[3];
        for (int c = 0; c < 3; c++) {
            // wrap into [0, L) and round to the fixed-point grid: one rounding per
            // operation (no contraction), so the conversion is reproducible
            double L = (double)d.Lq[c] * kInvFix;
            double x = d.io[3 * i + c];
            double fl = floor(__ddiv_rn(x, L));
            int im = (int)fl;
            double xw = __dsub_rn(x, __dmul_rn(fl, L));
            long long q = __double2ll_rn(__dmul_rn(xw, kFix));
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
            qs[c] = q;
        }
        int ty = d.io_int[i];
        if ((unsigned)ty >= (unsigned)d.ntypes) {  // (device input is not checked on the host)
            atomicOr(&d.ctl->status, kStatusBadType);
            ty = 0;
        }
        P4 p;
        p.x = snap_coord(qs[0], 0, d);
        p.y = snap_coord(qs[1], 1, d);
        p.z = snap_coord(qs[2], 2, d);
        p.w = snap_bits((i << kTypeBits) | ty, d);
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
        const int bits = pos_bits(d.pos[pc][q]);
        int tag = bits >> kTypeBits;
        R4 v = d.vel[ac][q];
        for (int c = 0; c < 3; c++) {
            d.io[3 * tag + c] = (double)d.xq[ac][c * n + q] * kInvFix;
            d.io_int[n + 3 * tag + c] = d.img[ac][c * n + q];
        }
        d.io[3 * n + 3 * tag + 0] = (double)v.x;
        d.io[3 * n + 3 * tag + 1] = (double)v.y;
        d.io[3 * n + 3 * tag + 2] = (double)v.z;
        d.io_int[tag] = bits & ((1 << kTypeBits) - 1);
    }
}

// pc < 0: the current snapshot set as the control block records it.
template <typename Real>
__global__ void k_get_forces(Dev<Real> d, int pc)
{
    typedef typename Dev<Real>::R4 R4;
    const int n = d.n;
    if (pc < 0) pc = d.ctl->pos_cur;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int tag = pos_bits(d.pos[pc][q]) >> kTypeBits;
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
        const int tag = pos_bits(d.pos[pc][q]) >> kTypeBits;
        const int4 inf = d.pinfo[q];
        counts[2 * tag] = inf.y;
        counts[2 * tag + 1] = inf.y + inf.w;
        int* out = rows + (size_t)tag * width;
        int k = 0;
        for (int e = inf.x; e < inf.x + inf.y && k < width; e++, k++)
            out[k] = pos_bits(d.pos[pc][d.ent_j[e]]) >> kTypeBits;
        for (int e = inf.z; e < inf.z + inf.w && k < width; e++, k++)
            out[k] = pos_bits(d.pos[pc][d.ent_j[e]]) >> kTypeBits;
    }
}

// ---------------------------------------------------------------------------
// Derivatives with respect to the reactive pair's coefficients (lambda, eps,
// sigma), at the current positions and list, for one reactive type pair
// (a^2 = lambda eps) and the unshifted form.  With x = (sigma/r)^n:
//   v = 4 eps (x^2 - x),  vh = 4 (x - x^2) beyond r_min (1 inside),
//   Q = 4 n (2x^2 - x) (= -r v'/eps), q = Q beyond r_min (0 inside) (= r vh'),
//   S_i = sum_k vh_ik, D_i = sum_k q_ik (over i's reactive partners inside r_cut),
//   T = sum_i sum_{j<k} vh_ij vh_ik = 1/2 sum_i (S_i^2 - sum_j vh_ij^2),
//   U = sum_pairs v + lambda eps T (+ the pairs that do not depend on theta).
// Then dU/dlambda = eps T, dU/deps = sum_pairs v/eps + lambda T,
//   dU/dsigma = (eps sum_pairs Q + lambda eps sum_i (sum_j vh_ij q_ij - S_i D_i)) / sigma,
// and, with the pair force F_i = -ft (x_j - x_i), ft = eps (Q - lambda g q) / r^2,
// g = S_i + S_j - 2 vh:
//   dft/dlambda = -eps g q / r^2,   dft/deps = (Q - lambda g q) / r^2,
//   dft/dsigma = (eps Q_s - lambda eps ((2q - D_i - D_j) q + g q_s)) / (sigma r^2),
//   Q_s = 4 n^2 x (4x - 1) (= sigma dQ/dsigma), q_s = Q_s beyond r_min (0 inside).
// Decisions (inside r_cut, beyond r_min) are the force kernels' own.

template <typename Real>
__device__ __forceinline__ Real pair_x(const PairP<Real>& p, Real r2)
{
    const Real s2 = p.sig2 * recip(r2);
    Real x = ipow(s2, p.nhalf);
    if (p.odd) x *= sqrt(s2);
    return x;
}

// The two passes give each particle kPgLanes consecutive lanes of a warp:
// lane l of the group takes the particle's reactive entries l, l + kPgLanes,
// ..., and the group's partial sums meet in a fixed shuffle tree, so the
// gathers of a particle's partners run in parallel (and the grid fills the
// device at a few 10^4 particles).
constexpr int kPgLanes = 4;

__device__ __forceinline__ double pg_group_sum(double v)
{
#pragma unroll
    for (int o = kPgLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, kPgLanes);
    return v;
}

// Pass 1: S_i and D_i per slot into sd[2i], sd[2i+1]; per-block sums of
// (T, sum_i (sum_j vh q - S D), sum_pairs v/eps, sum_pairs Q) into part[4b..].
template <typename Real>
__global__ void k_pgrad_sums(Dev<Real> d, int pc, double* sd, double* part)
{
    __shared__ double red[4][32];
    const int n = d.n;
    if (pc < 0) pc = d.ctl->pos_cur;
    const int g = threadIdx.x % kPgLanes;
    const int gpb = blockDim.x / kPgLanes;  // particles per block and round
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    // every lane of a warp runs the same number of rounds (the shuffles need them all)
    const int rounds = (n + gpb * gridDim.x - 1) / (gpb * gridDim.x);
    for (int r = 0; r < rounds; r++) {
        const int i = (r * gridDim.x + blockIdx.x) * gpb + (int)threadIdx.x / kPgLanes;
        double S = 0.0, D = 0.0, v2 = 0.0, vq = 0.0, ve = 0.0, qq = 0.0;
        if (i < n) {
            const typename Dev<Real>::P4 pi = d.pos[pc][i];
            const int4 inf = d.pinfo[i];
            for (int e = inf.x + g; e < inf.x + inf.y; e += kPgLanes) {
                const typename Dev<Real>::P4 pj = d.pos[pc][d.ent_j[e]];
                const PairP<Real>& p = d.table[type_of(pi) * d.ntypes + type_of(pj)];
                Real dx, dy, dz;
                const Real r2 = dist2_listed(pi, pj, d, dx, dy, dz);
                if (!(r2 < p.rc2)) continue;
                const double x = (double)pair_x(p, r2), nn = (double)p.n_real;
                const bool beyond = r2 > p.rmin2;
                const double vh = beyond ? 4.0 * (x - x * x) : 1.0;
                const double Q = 4.0 * nn * (2.0 * x * x - x);
                const double q = beyond ? Q : 0.0;
                S += vh;
                D += q;
                v2 += vh * vh;
                vq += vh * q;
                ve += 0.5 * 4.0 * (x * x - x);  // each pair is listed from both ends
                qq += 0.5 * Q;
            }
        }
        S = pg_group_sum(S);
        D = pg_group_sum(D);
        v2 = pg_group_sum(v2);
        vq = pg_group_sum(vq);
        ve = pg_group_sum(ve);
        qq = pg_group_sum(qq);
        if (i < n && g == 0) {
            sd[2 * i] = S;
            sd[2 * i + 1] = D;
            acc[0] += 0.5 * (S * S - v2);
            acc[1] += vq - S * D;
            acc[2] += ve;
            acc[3] += qq;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int k = 0; k < nw; k++) t += red[threadIdx.x][k];
        part[4 * blockIdx.x + threadIdx.x] = t;
    }
}

// Pass 2: dF/dtheta per particle, in user order: out[(k n + tag) 3 + c];
// theta = (lambda, eps, sigma) in device memory.
template <typename Real>
__global__ void k_pgrad_forces(Dev<Real> d, int pc, const double* sd, const double* theta, double* out)
{
    const int n = d.n;
    if (pc < 0) pc = d.ctl->pos_cur;
    const double lam = theta[0], eps = theta[1], sig = theta[2];
    const int g = threadIdx.x % kPgLanes;
    const int gpb = blockDim.x / kPgLanes;
    const int rounds = (n + gpb * gridDim.x - 1) / (gpb * gridDim.x);
    for (int r = 0; r < rounds; r++) {
        const int i = (r * gridDim.x + blockIdx.x) * gpb + (int)threadIdx.x / kPgLanes;
        double g3[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
        int tag = 0;
        if (i < n) {
            const typename Dev<Real>::P4 pi = d.pos[pc][i];
            const int4 inf = d.pinfo[i];
            const double Si = sd[2 * i], Di = sd[2 * i + 1];
            tag = pos_bits(pi) >> kTypeBits;
            for (int e = inf.x + g; e < inf.x + inf.y; e += kPgLanes) {
                const int j = d.ent_j[e];
                const typename Dev<Real>::P4 pj = d.pos[pc][j];
                const PairP<Real>& p = d.table[type_of(pi) * d.ntypes + type_of(pj)];
                Real dx, dy, dz;
                const Real r2 = dist2_listed(pi, pj, d, dx, dy, dz);
                if (!(r2 < p.rc2)) continue;
                const double x = (double)pair_x(p, r2), nn = (double)p.n_real, rr = (double)r2;
                const bool beyond = r2 > p.rmin2;
                const double vh = beyond ? 4.0 * (x - x * x) : 1.0;
                const double Q = 4.0 * nn * (2.0 * x * x - x);
                const double q = beyond ? Q : 0.0;
                const double Qs = 4.0 * nn * nn * x * (4.0 * x - 1.0);
                const double qs = beyond ? Qs : 0.0;
                const double gg = Si + sd[2 * j] - 2.0 * vh;
                const double Dsum = Di + sd[2 * j + 1];
                const double dft[3] = {-eps * gg * q / rr, (Q - lam * gg * q) / rr,
                                       (eps * Qs - lam * eps * ((2.0 * q - Dsum) * q + gg * qs)) / (sig * rr)};
                const double dv[3] = {(double)dx, (double)dy, (double)dz};
#pragma unroll
                for (int k = 0; k < 3; k++)
#pragma unroll
                    for (int c = 0; c < 3; c++) g3[k][c] -= dft[k] * dv[c];
            }
        }
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int c = 0; c < 3; c++) g3[k][c] = pg_group_sum(g3[k][c]);
        if (i < n && g < 3) {  // lanes 0..2 of the group write parameter k = g
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k == g)
#pragma unroll
                    for (int c = 0; c < 3; c++) out[((size_t)k * n + tag) * 3 + c] = g3[k][c];
        }
    }
}

// Pass 3: one block of four warps adds the per-block sums into total[4] --
// warp k sums quantity k, lane l the blocks l, l + 32, ... in order, then a
// fixed shuffle tree -- and forms dU/dtheta from them into dU[3] (when given).
static __global__ void k_pgrad_total(const double* part, int nblocks, double* total, const double* theta,
                                     double* dU)
{
    __shared__ double t[4];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k < 4) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) v += part[4 * b + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            total[k] = v;
            t[k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && dU) {
        // t = (T, sum_i (sum_j vh q - S D), sum_pairs v/eps, sum_pairs Q)
        const double lam = theta[0], eps = theta[1], sig = theta[2];
        dU[0] = eps * t[0];
        dU[1] = t[2] + lam * t[0];
        dU[2] = (eps * t[3] + lam * eps * t[1]) / sig;
    }
}

// Start of one device-driven evaluation (swp_eval_grad): resets the control
// block as a new state does (forces stale, list to be rebuilt), writes the
// reactive pair's coefficients from theta = (lambda, eps, sigma) in device
// memory into both (ti, tj) entries of the device pair table (the
// theta-dependent ones; the same arithmetic as the host table), and fills
// the state staging: velocities 0, masses 1, images 0, types from type.
// c_rmin = 2^(1/n), c_rb = ((1 - sqrt(1/2)) / 2)^(-1/n) (host constants),
// rbond > 0: the bond radius as given.
template <typename Real>
__global__ void k_eval_prep(Dev<Real> d, int ti, int tj, const double* theta, double c_rmin, double c_rb,
                            double rbond, const int* type)
{
    const int n = d.n;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl* ctl = d.ctl;
        int* w = (int*)ctl;
        for (int k = 0; k < (int)(sizeof(Ctl) / sizeof(int)); k++) w[k] = 0;
        ctl->state = 1;
        ctl->need_rebuild = 1;
        const double lam = theta[0], eps = theta[1], sig = theta[2];
        PairP<Real>* tab = (PairP<Real>*)d.table;
        PairP<Real> e = tab[ti * d.ntypes + tj];
        e.four_eps = (Real)(4.0 * eps);
        e.sig2 = (Real)(sig * sig);
        const double rmin = sig * c_rmin;
        e.rmin2 = (Real)(rmin * rmin);
        e.a = (Real)sqrt(lam * eps);
        e.inv_epshat = (Real)(1.0 / eps);
        const double rb = rbond > 0.0 ? rbond : sig * c_rb;
        e.rbond2 = (Real)(rb * rb);
        tab[ti * d.ntypes + tj] = e;
        tab[tj * d.ntypes + ti] = e;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; c++) {
            d.io[3 * n + 3 * i + c] = 0.0;
            d.io_int[n + 3 * i + c] = 0;
        }
        d.io[6 * n + i] = 1.0;
        d.io_int[i] = type ? type[i] : 0;
    }
}

#endif  // SWP_HAS_RESIDENT

}  // namespace single / wide / SWP_BATCH_NS
}  // namespace swp
