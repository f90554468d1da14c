// Host side of the C-ABI declared in include/swapmd.h: validation, the
// workspace layout, parameter tables, launches and the user-order exchange.
// The library allocates no device memory; everything lives in the caller's
// workspace and neighbour-list buffers.
#include "swapmd.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <utility>
#include <type_traits>
#include <vector>

#include "swp_internal.h"

using namespace swp;

namespace {

struct PairHost {
    int kind = KIND_NONE;
    int n = 6;
    int shift = 0;
    double eps = 1.0, sigma = 1.0, lambda3 = 0.0, rcut = 0.0, rbond = 0.0;
};

// Thermo-log record first + blockIdx.x (in ring slot (first + r) % cap): warp
// q sums quantity q of the block partials of the grid that wrote the record,
// in the order of the step kernel's end-of-launch reduction (32 blocks per
// shuffle tree, the trees' sums in block order), so a logged last step reads
// the same as the launch's thermo record.
__global__ void k_tlog_reduce(const double* ring, const long long* steps, int cap, int max_blocks,
                              long long first, double* out, long long* out_step)
{
    const long long r = blockIdx.x;
    const int slot = (int)((first + r) % cap);
    const int G = (int)steps[2 * slot + 1];
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* src = ring + (size_t)slot * max_blocks * kNQ + q;
    double t = 0.0;
    for (int w = 0; w < (G + 31) / 32; w++) {
        const int b = 32 * w + lane;
        double v = b < G ? src[(size_t)b * kNQ] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        t += v;
    }
    if (lane == 0) out[r * kNQA + q] = t;
    if (threadIdx.x == 0) out_step[r] = steps[2 * slot];
}

// End of the force part of a device-driven evaluation: U = U2 + U3 of the
// thermo record.
__global__ void k_eval_energy(const Ctl* ctl, double* U) { U[0] = ctl->thermo[Q_U2] + ctl->thermo[Q_U3]; }

__global__ void k_mark_stale(Ctl* ctl)
{
    if (ctl->state == 0) ctl->state = 1;
    ctl->need_rebuild = 1;
}

__global__ void k_clear_status_bits(Ctl* ctl, int bits) { ctl->status &= ~bits; }

}  // namespace

struct swp_ctx {
    int n = 0, ntypes = 1, precision = SWP_FP32;
    double box[3] = {0, 0, 0};
    uint64_t seed = 0;
    double skin = 0.3;
    int max_nn = 64;
    PairHost pairs[kMaxTypes * kMaxTypes];
    int nc[3] = {3, 3, 3};
    int ncell = 27;
    int device = 0, num_sms = 0;
    int bps_req = 0, grid_req = 0, grid = 0, max_blocks = 0;
    long long timeout_ns = 2000000000LL;
    int resident = 1;  // the FP32 step may keep each block's neighbourhood in shared memory
    int withhold = 0;  // test hook: the next launch withholds one barrier arrival
    int tlog_every = 0;  // thermo log: every how many steps a record is written (0: off)
    int table_only = 0;      // the next launch reads pair coefficients from the device table (not the uniform copy)
    bool table_theta = false;  // swp_eval_grad wrote theta's coefficients into the device table
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* nl = nullptr;
    size_t nl_bytes = 0;
    cudaStream_t stream = nullptr;
    bool ws_bound = false, nl_bound = false, state_set = false, table_dirty = true;
    bool layout_dirty = true;
    std::vector<int> bond_host;  // [n][kMaxBonds] partner tags by tag (-1: none); empty: no bonds
    double bond_k = 0.0, bond_r0 = 1.0;
    bool bonds_dirty = false;
    Dev<float> df;
    Dev<double> dd;
    Ctl hctl;
    std::vector<int> cell_rank;
    std::vector<unsigned char> table_host;
    std::string err;
};

namespace {

int fail(swp_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(swp_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, SWP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SWP_CUDA(c, call)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call);   \
    } while (0)

double pair_cut(const PairHost& p)
{
    if (p.kind == KIND_WCA) return p.sigma * std::pow(2.0, 1.0 / p.n);
    if (p.kind == KIND_SWAP) return p.rcut;
    return 0.0;
}

double lj(double r, double eps, double sigma, int n)
{
    double x = std::pow(sigma / r, (double)n);
    return 4.0 * eps * (x * x - x);
}

double max_list_radius(const swp_ctx* c)
{
    double m = 0.0;
    for (int t = 0; t < c->ntypes * c->ntypes; t++) {
        double cut = pair_cut(c->pairs[t]);
        if (cut > 0.0) m = std::max(m, cut + c->skin);
    }
    return m;
}

unsigned long long spread3(unsigned v)
{
    unsigned long long x = v & 0x3ff;
    unsigned long long r = 0;
    for (int b = 0; b < 10; b++) r |= ((x >> b) & 1ull) << (3 * b);
    return r;
}

// Cell grid and its Morton order (cells that are close in space are close
// in the sorted particle arrays, so neighbour gathers share cache lines).
int derive_cells(swp_ctx* c)
{
    double rl = max_list_radius(c);
    for (int d = 0; d < 3; d++) {
        int k = rl > 0.0 ? (int)std::floor(c->box[d] / (rl * (1.0 + 1e-5))) : 3;
        if (rl > 0.0 && k < 3)
            return fail(c, SWP_ERR_INVALID,
                        "box too small: each box length must hold 3 cells of edge max(cut-off) + skin");
        c->nc[d] = std::max(3, std::min(k, 1024));
    }
    long long nce = (long long)c->nc[0] * c->nc[1] * c->nc[2];
    if (nce > (1LL << 30)) return fail(c, SWP_ERR_INVALID, "too many cells");
    c->ncell = (int)nce;
    std::vector<std::pair<unsigned long long, int>> code(c->ncell);
    for (int z = 0; z < c->nc[2]; z++)
        for (int y = 0; y < c->nc[1]; y++)
            for (int x = 0; x < c->nc[0]; x++) {
                int lin = (z * c->nc[1] + y) * c->nc[0] + x;
                code[lin] = {spread3(x) | (spread3(y) << 1) | (spread3(z) << 2), lin};
            }
    std::sort(code.begin(), code.end());
    c->cell_rank.assign(2 * (size_t)c->ncell, 0);
    for (int r = 0; r < c->ncell; r++) {
        c->cell_rank[code[r].second] = r;
        c->cell_rank[c->ncell + r] = code[r].second;
    }
    return SWP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Neighbour-list buffer: entries of every block's region (capacity
// (n + max_blocks) * max_nn, enough for any grid of at most max_blocks
// blocks): partner slots, then owner indices (both int32).
size_t list_entries(const swp_ctx* c) { return ((size_t)std::max(c->n, 1) + c->max_blocks) * c->max_nn; }

size_t list_bytes(const swp_ctx* c) { return align256(list_entries(c) * 4) + align256(list_entries(c) * 2); }

template <typename Real>
void set_list(const swp_ctx* c, char* base, Dev<Real>* d)
{
    d->ent_j = (int*)base;
    d->ent_o = base ? (unsigned short*)(base + align256(list_entries(c) * 4)) : nullptr;
}

// Carves the workspace; with base == nullptr only measures it.
template <typename Real>
size_t layout(swp_ctx* c, char* base, Dev<Real>* d)
{
    typedef typename Dev<Real>::R4 R4;
    const size_t n = (size_t)std::max(c->n, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return base ? base + o : nullptr;
    };
    Ctl* ctl = (Ctl*)take(sizeof(Ctl));
    PairP<Real>* table = (PairP<Real>*)take(sizeof(PairP<Real>) * kMaxTypes * kMaxTypes);
    typedef typename Dev<Real>::P4 P4;
    P4* pos0 = (P4*)take(sizeof(P4) * n);
    P4* pos1 = (P4*)take(sizeof(P4) * n);
    long long* xq0 = (long long*)take(sizeof(long long) * 3 * n);
    long long* xq1 = (long long*)take(sizeof(long long) * 3 * n);
    int* img0 = (int*)take(sizeof(int) * 3 * n);
    int* img1 = (int*)take(sizeof(int) * 3 * n);
    R4* vel0 = (R4*)take(sizeof(R4) * n);
    R4* vel1 = (R4*)take(sizeof(R4) * n);
    R4* force = (R4*)take(sizeof(R4) * n);
    Real* S = (Real*)take(sizeof(Real) * n);
    int4* pinfo = (int4*)take(sizeof(int4) * n);
    int* cell_rank = (int*)take(sizeof(int) * 2 * c->ncell);
    int* cell_cnt = (int*)take(sizeof(int) * c->ncell);
    int* cell_start = (int*)take(sizeof(int) * (c->ncell + 1));
    int* cell_fill = (int*)take(sizeof(int) * (c->ncell + n));
    int* perm = (int*)take(sizeof(int) * n);
    int* bsum = (int*)take(sizeof(int) * c->max_blocks);
    // thermo partials of the step kernel; also the scratch of the parameter derivatives (4 * 512 + 16)
    double* partials = (double*)take(sizeof(double) * std::max<size_t>((size_t)c->max_blocks * kNQ, 4 * 512 + 16));
    double* io = (double*)take(sizeof(double) * 7 * n);
    int* io_int = (int*)take(sizeof(int) * 4 * n);
    int* bond_tag = (int*)take(sizeof(int) * kMaxBonds * n);
    int* slot_of_tag = (int*)take(sizeof(int) * n);
    if (d) {
        d->n = c->n;
        d->ntypes = c->ntypes;
        d->max_nn = c->max_nn;
        d->ncell = c->ncell;
        for (int k = 0; k < 3; k++) {
            d->nc[k] = c->nc[k];
            long long q = (long long)std::llround(c->box[k] * kFix);
            d->Lq[k] = q;
            double L = (double)q * kInvFix;
            d->L[k] = (Real)L;
            d->hL[k] = (Real)(0.5 * (double)(Real)L);
            d->inv_cw[k] = (Real)(c->nc[k] / L);
            d->iL[k] = (Real)(1.0 / (double)(Real)L);
            d->fmul[k] = (unsigned long long)(((unsigned __int128)1 << 96) / (unsigned __int128)q);
            d->fscale[k] = (float)((double)q * 0x1p-80);
        }
        d->pos[0] = pos0;
        d->pos[1] = pos1;
        d->xq[0] = xq0;
        d->xq[1] = xq1;
        d->img[0] = img0;
        d->img[1] = img1;
        d->vel[0] = vel0;
        d->vel[1] = vel1;
        d->force = force;
        d->S = S;
        set_list(c, (char*)c->nl, d);
        d->pinfo = pinfo;
        d->cell_rank = cell_rank;
        d->cell_cnt = cell_cnt;
        d->cell_start = cell_start;
        d->cell_fill = cell_fill;
        d->perm = perm;
        d->bsum = bsum;
        d->partials = partials;
        d->ctl = ctl;
        d->io = io;
        d->io_int = io_int;
        d->table = table;
        d->bond_tag = bond_tag;
        d->slot_of_tag = slot_of_tag;
        d->has_bonds = 0;  // set per run (prepare_args) when bonds were given
        d->bond_k = Real(0);
        d->bond_r0 = Real(1);
    }
    return off;
}

size_t workspace_bytes(swp_ctx* c)
{
    return c->precision == SWP_FP64 ? layout<double>(c, nullptr, nullptr)
                                    : layout<float>(c, nullptr, nullptr);
}

// Every type pair's device coefficients (precomputed in double, stored in the
// run's precision): the one place the table is derived from the context.
template <typename Real>
void fill_pair_table(const swp_ctx* c, PairP<Real>* t)
{
    std::memset(t, 0, sizeof(PairP<Real>) * kMaxTypes * kMaxTypes);
    for (int k = 0; k < c->ntypes * c->ntypes; k++) {
        const PairHost& p = c->pairs[k];
        PairP<Real> e;
        std::memset(&e, 0, sizeof(e));
        e.kind = p.kind;
        e.nhalf = p.n / 2;
        e.odd = p.n & 1;
        e.four_eps = (Real)(4.0 * p.eps);
        e.n_real = (Real)p.n;
        e.sig2 = (Real)(p.sigma * p.sigma);
        const double rmin = p.sigma * std::pow(2.0, 1.0 / p.n);
        e.rmin2 = (Real)(rmin * rmin);
        e.rlist2 = (Real)(-1.0);
        if (p.kind == KIND_WCA) {
            e.rc2 = (Real)(rmin * rmin);
            e.ushift = (Real)p.eps;
            e.inv_epshat = (Real)(1.0 / p.eps);
            e.rlist2 = (Real)((rmin + c->skin) * (rmin + c->skin));
            e.rbond2 = (Real)(-1.0);
        } else if (p.kind == KIND_SWAP) {
            const double vc = p.shift ? lj(p.rcut, p.eps, p.sigma, p.n) : 0.0;
            e.rc2 = (Real)(p.rcut * p.rcut);
            e.a = (Real)std::sqrt(p.lambda3 * p.eps);
            e.inv_epshat = (Real)(1.0 / (p.eps + vc));
            e.vshift = (Real)vc;
            e.ushift = (Real)(-vc);
            e.rlist2 = (Real)((p.rcut + c->skin) * (p.rcut + c->skin));
            double rb = p.rbond > 0.0 ? p.rbond
                                      : p.sigma * std::pow((1.0 - std::sqrt(0.5)) / 2.0, -1.0 / p.n);
            e.rbond2 = (Real)(rb * rb);
        }
        t[k] = e;
    }
}

template <typename Real>
void build_table(swp_ctx* c)
{
    c->table_host.assign(sizeof(PairP<Real>) * kMaxTypes * kMaxTypes, 0);
    fill_pair_table<Real>(c, (PairP<Real>*)c->table_host.data());
}

template <typename Real>
Dev<Real>& dev(swp_ctx* c);
template <>
Dev<float>& dev<float>(swp_ctx* c) { return c->df; }
template <>
Dev<double>& dev<double>(swp_ctx* c) { return c->dd; }

int refresh_layout(swp_ctx* c)
{
    if (!c->ws_bound) return fail(c, SWP_ERR_STATE, "no workspace bound");
    if (c->precision == SWP_FP64) layout<double>(c, (char*)c->ws, &c->dd);
    else layout<float>(c, (char*)c->ws, &c->df);
    if (c->precision == SWP_FP64) set_list(c, (char*)c->nl, &c->dd);
    else set_list(c, (char*)c->nl, &c->df);
    c->bonds_dirty = !c->bond_host.empty();  // the bond table moved with the layout
    return SWP_OK;
}

Ctl* dev_ctl(swp_ctx* c) { return c->precision == SWP_FP64 ? c->dd.ctl : c->df.ctl; }

int upload_table(swp_ctx* c)
{
    if (!c->table_dirty) return SWP_OK;
    void* dst;
    if (c->precision == SWP_FP64) {
        build_table<double>(c);
        dst = (void*)c->dd.table;
    } else {
        build_table<float>(c);
        dst = (void*)c->df.table;
    }
    SWP_CUDA(c, cudaMemcpyAsync(dst, c->table_host.data(), c->table_host.size(),
                                cudaMemcpyHostToDevice, c->stream));
    c->table_dirty = false;
    return SWP_OK;
}

int ready(swp_ctx* c, bool need_state)
{
    if (!c) return SWP_ERR_INVALID;
    if (!c->ws_bound) return fail(c, SWP_ERR_STATE, "no workspace bound");
    if (!c->nl_bound && c->n > 0) return fail(c, SWP_ERR_STATE, "no neighbour-list buffer bound");
    if (need_state && !c->state_set) return fail(c, SWP_ERR_STATE, "no state set");
    return SWP_OK;
}

int map_status(swp_ctx* c)
{
    int s = c->hctl.status;
    if (s & kStatusTimeout) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "a device-side wait timed out (phase %lld); set the state again",
                      c->hctl.timeout_at);
        return fail(c, SWP_ERR_TIMEOUT, buf);
    }
    if (s & kStatusBadType) return fail(c, SWP_ERR_INVALID, "a particle type is out of range; set the state again");
    if (s & kStatusNonfinite) return fail(c, SWP_ERR_NONFINITE, "non-finite force; set the state again");
    if (s & kStatusOverflow) {
        cudaError_t e = cudaSuccess;
        k_clear_status_bits<<<1, 1, 0, c->stream>>>(dev_ctl(c), kStatusOverflow);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "clear status");
        char buf[160];
        std::snprintf(buf, sizeof buf, "neighbour row of %d entries exceeds max_nn = %d",
                      c->hctl.max_row, c->max_nn);
        return fail(c, SWP_ERR_NLIST_OVERFLOW, buf);
    }
    return SWP_OK;
}

// Waits for the stream and refreshes the host copy of the control block.
int sync_ctl(swp_ctx* c)
{
    if (c->n == 0 || !c->state_set) {
        SWP_CUDA(c, cudaStreamSynchronize(c->stream));
        return SWP_OK;
    }
    SWP_CUDA(c, cudaMemcpyAsync(&c->hctl, dev_ctl(c), sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    return map_status(c);
}

template <typename Real>
PairP<Real>* uni_slot(RunArgs* a);
template <>
PairP<float>* uni_slot<float>(RunArgs* a) { return a->uf; }
template <>
PairP<double>* uni_slot<double>(RunArgs* a) { return a->ud; }

bool same_pair(const PairHost& a, const PairHost& b)
{
    return a.kind == b.kind && a.n == b.n && a.shift == b.shift && a.eps == b.eps &&
           a.sigma == b.sigma && a.lambda3 == b.lambda3 && a.rcut == b.rcut && a.rbond == b.rbond;
}

// Uniform coefficients: one parameter set for every reactive pair and one for
// every other interacting pair lets the kernels keep them in registers.
void uniform_pairs(const swp_ctx* c, RunArgs* a)
{
    int sw = -1, ot = -1;
    bool uni = true;
    for (int k = 0; k < c->ntypes * c->ntypes; k++) {
        const PairHost& p = c->pairs[k];
        if (p.kind == KIND_SWAP) {
            if (sw < 0) sw = k;
            else if (!same_pair(p, c->pairs[sw])) uni = false;
        } else if (p.kind == KIND_WCA) {
            if (ot < 0) ot = k;
            else if (!same_pair(p, c->pairs[ot])) uni = false;
        }
    }
    a->uni = uni ? 1 : 0;
    a->uni_swap = sw < 0 ? 0 : sw;
    a->uni_other = ot < 0 ? 0 : ot;
}

// Fills the system-dependent run arguments (table upload included).
template <typename Real>
int prepare_args(swp_ctx* c, RunArgs& a)
{
    int rc = upload_table(c);
    if (rc) return rc;
    Dev<Real>& dv = dev<Real>(c);
    if (c->bonds_dirty) {
        SWP_CUDA(c, cudaMemcpyAsync(dv.bond_tag, c->bond_host.data(), sizeof(int) * c->bond_host.size(),
                                    cudaMemcpyHostToDevice, c->stream));
        c->bonds_dirty = false;
    }
    dv.has_bonds = c->bond_host.empty() ? 0 : 1;
    dv.bond_k = (Real)c->bond_k;
    dv.bond_r0 = (Real)c->bond_r0;
    a.max_blocks = c->max_blocks;
    a.timeout_ns = c->timeout_ns;
    double margin = 0.0;
    if (c->precision == SWP_FP32) {
        double Lm = std::max(c->box[0], std::max(c->box[1], c->box[2]));
        margin = 8.0 * Lm * std::ldexp(1.0, -24);
    }
    a.skin_eff = c->skin - margin;
    a.seed = c->seed;
    uniform_pairs(c, &a);
    if (a.uni) {
        const PairP<Real>* t = (const PairP<Real>*)c->table_host.data();
        PairP<Real>* u = uni_slot<Real>(&a);
        u[0] = t[a.uni_swap];
        u[1] = t[a.uni_other];
    }
    return SWP_OK;
}

// Blocks of the step kernel: the resident blocks of every SM, or fewer on
// request, but at least kNQA (the thermo quantities are reduced one per block).
int step_grid(const swp_ctx* c, int bps)
{
    const int g = c->num_sms * bps;
    return c->grid_req > 0 ? std::min(g, std::max(c->grid_req, kNQA)) : g;
}

template <typename Real>
int run(swp_ctx* c, RunArgs a)
{
    Dev<Real>& d = dev<Real>(c);
    int bps = 0;
    SWP_CUDA(c, run_occupancy<Real>(kBlock, &bps));
    if (bps < 1) return fail(c, SWP_ERR_CUDA, "step kernel does not fit on an SM");
    if (c->bps_req > 0) bps = std::min(bps, c->bps_req);
    bps = std::min(bps, c->max_blocks / std::max(c->num_sms, 1));
    c->grid = step_grid(c, bps);
    // a bonded network runs the 1024-thread kernel (two-barrier step: more
    // warps hide its global gathers; 434 against 500 us per step on the 2M-bead
    // network), everything else the 768-thread one (the resident step where it
    // applies; at 1M-2M unbonded particles the two shapes are within 3 %, the
    // 768-thread one ahead)
    const bool wide = !c->bond_host.empty();
    if (wide) {
        int bw = 0;
        SWP_CUDA(c, run_occupancy_wide<Real>(&bw));
        if (bw < 1) return fail(c, SWP_ERR_CUDA, "step kernel does not fit on an SM");
        if (c->bps_req > 0) bw = std::min(bw, c->bps_req);
        bw = std::min(bw, c->max_blocks / std::max(c->num_sms, 1));
        c->grid = step_grid(c, bw);
    }
    if (!c->table_only && c->table_theta) {  // an ordinary run takes the host coefficients again
        c->table_dirty = true;
        c->table_theta = false;
    }
    int rc = prepare_args<Real>(c, a);
    if (rc) return rc;
    a.resident = c->resident;
    a.withhold = c->withhold;
    a.tlog_every = d.tlog ? c->tlog_every : 0;
    if (c->table_only) a.uni = 0;  // the device table holds coefficients the host copy does not
    c->withhold = 0;  // one launch consumes the request
    SWP_CUDA(c, cudaMemsetAsync(&d.ctl->barrier, 0, sizeof(unsigned long long), c->stream));
    if (wide) SWP_CUDA(c, launch_run_wide<Real>(d, a, c->grid, c->stream));
    else SWP_CUDA(c, launch_run<Real>(d, a, c->grid, kBlock, c->stream));
    return SWP_OK;
}

int run_any(swp_ctx* c, RunArgs a)
{
    return c->precision == SWP_FP64 ? run<double>(c, a) : run<float>(c, a);
}

int mark_stale(swp_ctx* c)
{
    if (!c->ws_bound || !c->state_set || c->n == 0) return SWP_OK;
    k_mark_stale<<<1, 1, 0, c->stream>>>(dev_ctl(c));
    SWP_CUDA(c, cudaGetLastError());
    return SWP_OK;
}

cudaMemcpyKind kind_to_dev(int where)
{
    return where == SWP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

cudaMemcpyKind kind_from_dev(int where)
{
    return where == SWP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// ---------------------------------------------------------------------------
// Batched runs: m systems advanced by one cooperative launch of B blocks.
//
// The work of a system is taken as its particle count w; a block's load is
// the work of its items (a group member: w / group size).
//
// Balanced plan (split = 0): the smallest largest load C (bisection) for which
// every system heavier than C gets g = ceil(w / C) blocks (at most gmax, and
// no member share below min_part particles) with w / g <= C, and the other
// systems, heaviest first, each go onto the block with the least load so far
// (longest-processing-time rule; group members included, after their share)
// with no load above C.  A block runs its group share first, then its
// single-block systems: the members of a group start it together (every block
// of the cooperative launch is resident), so no group barrier waits for a
// block that is busy with another system.
//
// Threshold plan (split > 0): with T = sum(w) / B the mean load, a system
// heavier than split * T gets a group of max(1, round(w / T)) blocks of its
// own; the others are packed by the same rule onto the remaining blocks.
// Blocks left over when there is nothing to pack go to the groups with the
// most work per block.

struct BatchPlan {
    std::vector<int> item_ofs;  // [B + 1]
    std::vector<int4> items;    // (system, rank, group size, 0)
};

void plan_flatten(const std::vector<std::vector<int4>>& per, BatchPlan& plan)
{
    const int B = (int)per.size();
    plan.item_ofs.assign(B + 1, 0);
    plan.items.clear();
    for (int k = 0; k < B; k++) {
        plan.item_ofs[k] = (int)plan.items.size();
        for (const int4& it : per[k]) plan.items.push_back(it);
    }
    plan.item_ofs[B] = (int)plan.items.size();
}

// Whether the balanced plan fits under the largest load C; fills per if so.
// order: the systems heaviest first (ties by index).
bool plan_balanced_at(const std::vector<long long>& w, const std::vector<int>& order, int B, double C,
                      int gmax, int min_part, std::vector<std::vector<int4>>* per)
{
    std::vector<int> g(w.size(), 0);
    long long used = 0;
    for (int r : order) {
        const double x = (double)std::max(w[r], 1LL);
        if (x <= C) break;
        long long k = (long long)std::ceil(x / C);
        k = std::min<long long>(k, gmax);
        k = std::min<long long>(k, std::max<long long>(1, w[r] / std::max(min_part, 1)));
        if (x / (double)k > C) return false;
        g[r] = (int)k;
        used += k;
        if (used > B) return false;
    }
    if (per) per->assign(B, {});
    std::vector<std::pair<double, int>> heap;  // (load, block), least first
    heap.reserve(B);
    int b = 0;
    for (int r : order) {
        if (g[r] == 0) break;
        for (int k = 0; k < g[r]; k++, b++) {
            heap.push_back({(double)w[r] / g[r], b});
            if (per) (*per)[b].push_back(make_int4(r, k, g[r], 0));
        }
    }
    for (; b < B; b++) heap.push_back({0.0, b});
    std::make_heap(heap.begin(), heap.end(), std::greater<std::pair<double, int>>());
    for (int r : order) {
        if (g[r] > 0) continue;
        std::pop_heap(heap.begin(), heap.end(), std::greater<std::pair<double, int>>());
        std::pair<double, int>& top = heap.back();
        top.first += (double)std::max(w[r], 1LL);
        if (top.first > C) return false;
        if (per) (*per)[top.second].push_back(make_int4(r, 0, 1, 0));
        std::push_heap(heap.begin(), heap.end(), std::greater<std::pair<double, int>>());
    }
    return true;
}

int plan_balanced(const std::vector<long long>& w, int B, int gmax, int min_part, BatchPlan& plan)
{
    const int m = (int)w.size();
    std::vector<int> order(m);
    for (int r = 0; r < m; r++) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
    double W = 0.0;
    for (long long x : w) W += (double)std::max(x, 1LL);
    // hi always fits (no group, every load at most the total); lo is a bound
    double lo = W / B, hi = std::max(W, 1.0);
    std::vector<std::vector<int4>> per;
    if (plan_balanced_at(w, order, B, lo, gmax, min_part, &per)) {
        plan_flatten(per, plan);
        return 0;
    }
    for (int it = 0; it < 100 && hi > lo * (1.0 + 1e-6); it++) {
        const double mid = 0.5 * (lo + hi);
        if (plan_balanced_at(w, order, B, mid, gmax, min_part, nullptr))
            hi = mid;
        else
            lo = mid;
    }
    if (!plan_balanced_at(w, order, B, hi, gmax, min_part, &per)) return -1;
    plan_flatten(per, plan);
    return 0;
}

// gmax: the largest group (blocks given to one system); min_part: the
// smallest member share of a group in the balanced plan.
int plan_batch(const std::vector<long long>& w, int B, double split, int gmax, int min_part, BatchPlan& plan)
{
    if (split <= 0.0) return plan_balanced(w, B, gmax, min_part, plan);
    const int m = (int)w.size();
    long long W = 0;
    for (long long x : w) W += std::max(x, 1LL);
    const double T = (double)W / B;
    std::vector<int> g(m, 0);
    int used = 0;
    std::vector<int> order(m);
    for (int r = 0; r < m; r++) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
    for (int r : order)
        if ((double)w[r] > split * T) {
            g[r] = std::min(gmax, std::max(1, (int)std::llround((double)w[r] / T)));
            used += g[r];
        }
    bool small = false;
    for (int r = 0; r < m; r++) small |= g[r] == 0;
    const int need = small ? 1 : 0;
    // too many dedicated blocks: take them back from the groups with the least work per block
    while (used > B - need) {
        int best = -1;
        for (int r = 0; r < m; r++)
            if (g[r] > 1 && (best < 0 || (double)w[r] / g[r] < (double)w[best] / g[best])) best = r;
        if (best < 0) break;
        g[best]--;
        used--;
    }
    if (used > B - need) return -1;  // more heavy systems than blocks
    // nothing to pack: spread the spare blocks over the groups
    if (!small)
        while (used < B) {
            int best = -1;
            for (int r = 0; r < m; r++)
                if (g[r] > 0 && g[r] < gmax && (best < 0 || (double)w[r] / g[r] > (double)w[best] / g[best]))
                    best = r;
            if (best < 0) break;
            g[best]++;
            used++;
        }
    std::vector<std::vector<int4>> per(B);
    int b = 0;
    for (int r : order)
        if (g[r] > 0) {
            for (int k = 0; k < g[r]; k++) per[b + k].push_back(make_int4(r, k, g[r], 0));
            b += g[r];
        }
    const int first_free = b;
    std::vector<double> load(B, 0.0);
    for (int r : order)
        if (g[r] == 0) {
            int best = first_free;
            for (int k = first_free; k < B; k++)
                if (load[k] < load[best]) best = k;
            per[best].push_back(make_int4(r, 0, 1, 0));
            load[best] += (double)std::max(w[r], 1LL);
        }
    plan_flatten(per, plan);
    return 0;
}

size_t batch_bytes(int m, size_t dev_size)
{
    return align256(dev_size * m) + align256(sizeof(RunArgs) * m) + align256(sizeof(int) * (kMaxGrid + 1)) +
           align256(sizeof(int4) * (m + kMaxGrid));
}

// The block shapes of the batched kernel: 1024 threads in both precisions,
// 512, 384 and 256 in FP32.
bool batch_shape_ok(int precision, int threads)
{
    return threads == 1024 || (precision == SWP_FP32 && (threads == 512 || threads == 384 || threads == 256));
}

template <typename Real>
cudaError_t batch_occupancy_shape(int threads, int* bps)
{
    if constexpr (std::is_same<Real, float>::value) {
        if (threads == 512) return batch_occupancy_512(Prec<float>(), bps);
        if (threads == 384) return batch_occupancy_384(Prec<float>(), bps);
        if (threads == 256) return batch_occupancy_256(Prec<float>(), bps);
    }
    return batch_occupancy_1024(Prec<Real>(), bps);
}

template <typename Real>
cudaError_t launch_batch_shape(int threads, const Dev<Real>* devs, const RunArgs* args, const int* ofs,
                               const int4* items, int uni, int bonds, int grid, cudaStream_t s)
{
    if constexpr (std::is_same<Real, float>::value) {
        if (threads == 512) return launch_batch_512(devs, args, ofs, items, uni, bonds, grid, s);
        if (threads == 384) return launch_batch_384(devs, args, ofs, items, uni, bonds, grid, s);
        if (threads == 256) return launch_batch_256(devs, args, ofs, items, uni, bonds, grid, s);
    }
    return launch_batch_1024(devs, args, ofs, items, uni, bonds, grid, s);
}

template <typename Real>
int batch_run(swp_ctx* const* cs, const std::vector<int>& idx, std::vector<RunArgs>& args, double split,
              int threads, void* ws, size_t ws_bytes)
{
    swp_ctx* c0 = cs[idx[0]];
    const int m = (int)idx.size();
    int bps = 0;
    SWP_CUDA(c0, batch_occupancy_shape<Real>(threads, &bps));
    if (bps < 1) return fail(c0, SWP_ERR_CUDA, "batched step kernel does not fit on an SM");
    const int B = std::min(kMaxGrid, c0->num_sms * std::min(bps, 2048 / threads));
    if (ws_bytes < batch_bytes(m, sizeof(Dev<Real>))) return fail(c0, SWP_ERR_INVALID, "batch workspace too small");
    std::vector<long long> w(m);
    int gmax = threads;  // a group's thermo partials are reduced by one block's threads
    for (int r = 0; r < m; r++) {
        w[r] = cs[idx[r]]->n;
        gmax = std::min(gmax, cs[idx[r]]->max_blocks);  // and fit each system's partials
    }
    BatchPlan plan;
    if (plan_batch(w, B, split, gmax, threads, plan)) return fail(c0, SWP_ERR_INVALID, "more large systems than blocks");
    std::vector<Dev<Real>> devs(m);
    int uni = 1, bonds = 0;
    for (int r = 0; r < m; r++) {
        swp_ctx* c = cs[idx[r]];
        int rc = prepare_args<Real>(c, args[r]);
        if (rc) return rc;
        args[r].withhold = c->withhold;
        c->withhold = 0;  // one launch consumes the request
        uni &= args[r].uni;
        devs[r] = dev<Real>(c);
        bonds |= devs[r].has_bonds;
        SWP_CUDA(c0, cudaMemsetAsync(&devs[r].ctl->barrier, 0, sizeof(unsigned long long), c0->stream));
    }
    for (int k = 0; k < B; k++)
        for (int it = plan.item_ofs[k]; it < plan.item_ofs[k + 1]; it++)
            cs[idx[plan.items[it].x]]->grid = plan.items[it].z;
    char* base = (char*)ws;
    Dev<Real>* d_dev = (Dev<Real>*)base;
    RunArgs* d_args = (RunArgs*)(base + align256(sizeof(Dev<Real>) * m));
    int* d_ofs = (int*)((char*)d_args + align256(sizeof(RunArgs) * m));
    int4* d_items = (int4*)((char*)d_ofs + align256(sizeof(int) * (kMaxGrid + 1)));
    // pageable host sources: each copy has read its source when the call returns
    SWP_CUDA(c0, cudaMemcpyAsync(d_dev, devs.data(), sizeof(Dev<Real>) * m, cudaMemcpyHostToDevice, c0->stream));
    SWP_CUDA(c0, cudaMemcpyAsync(d_args, args.data(), sizeof(RunArgs) * m, cudaMemcpyHostToDevice, c0->stream));
    SWP_CUDA(c0, cudaMemcpyAsync(d_ofs, plan.item_ofs.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice,
                                 c0->stream));
    SWP_CUDA(c0, cudaMemcpyAsync(d_items, plan.items.data(), sizeof(int4) * plan.items.size(),
                                 cudaMemcpyHostToDevice, c0->stream));
    SWP_CUDA(c0, launch_batch_shape<Real>(threads, d_dev, d_args, d_ofs, d_items, uni, bonds, B, c0->stream));
    return SWP_OK;
}

}  // namespace

extern "C" {

int swp_abi_version(void) { return SWP_ABI_VERSION; }

int swp_create(swp_ctx** out, int n, int n_types, const double box[3], int precision,
               uint64_t seed)
{
    if (!out) return SWP_ERR_INVALID;
    *out = nullptr;
    if (n < 0 || n >= kMaxTag || n_types < 1 || n_types > kMaxTypes || !box) return SWP_ERR_INVALID;
    if (precision != SWP_FP32 && precision != SWP_FP64) return SWP_ERR_INVALID;
    for (int k = 0; k < 3; k++)
        if (!(box[k] >= 0x1p-8) || !std::isfinite(box[k]) || box[k] > 30000.0) return SWP_ERR_INVALID;
    swp_ctx* c = new swp_ctx();
    c->n = n;
    c->ntypes = n_types;
    c->precision = precision;
    c->seed = seed;
    for (int k = 0; k < 3; k++)
        c->box[k] = precision == SWP_FP32 ? (double)(float)box[k] : box[k];
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return SWP_ERR_CUDA;
    }
    c->max_blocks = std::min(kMaxGrid, c->num_sms * std::max(1, 2048 / kBlock));
    std::memset(&c->hctl, 0, sizeof(Ctl));
    if (derive_cells(c) != SWP_OK) {
        delete c;
        return SWP_ERR_INVALID;
    }
    *out = c;
    return SWP_OK;
}

int swp_set_pair(swp_ctx* c, int ti, int tj, int kind, double eps, double sigma, int n_exp,
                 double rcut, double lambda3, int shift, double rbond)
{
    if (!c) return SWP_ERR_INVALID;
    if (ti < 0 || tj < 0 || ti >= c->ntypes || tj >= c->ntypes)
        return fail(c, SWP_ERR_INVALID, "type index out of range");
    if (kind != KIND_NONE && kind != KIND_WCA && kind != KIND_SWAP)
        return fail(c, SWP_ERR_INVALID, "unknown pair kind");
    PairHost p;
    p.kind = kind;
    if (kind != KIND_NONE) {
        if (!(eps > 0.0) || !(sigma > 0.0) || n_exp < 1 || n_exp > 128 || !std::isfinite(eps) ||
            !std::isfinite(sigma))
            return fail(c, SWP_ERR_INVALID, "need eps > 0, sigma > 0, 1 <= n <= 128");
        p.eps = eps;
        p.sigma = sigma;
        p.n = n_exp;
    }
    if (kind == KIND_SWAP) {
        if (!(rcut > 0.0) || !std::isfinite(rcut) || !(lambda3 >= 0.0) || !std::isfinite(lambda3))
            return fail(c, SWP_ERR_INVALID, "need r_cut > 0 and lambda >= 0");
        if (shift != 0 && shift != 1) return fail(c, SWP_ERR_INVALID, "shift must be 0 or 1");
        if (shift && !(eps + lj(rcut, eps, sigma, n_exp) > 0.0))
            return fail(c, SWP_ERR_INVALID, "shifted form needs eps + v(r_cut) > 0");
        p.rcut = rcut;
        p.lambda3 = lambda3;
        p.shift = shift;
        p.rbond = std::isfinite(rbond) ? rbond : 0.0;
    }
    PairHost old_a = c->pairs[ti * c->ntypes + tj], old_b = c->pairs[tj * c->ntypes + ti];
    c->pairs[ti * c->ntypes + tj] = p;
    c->pairs[tj * c->ntypes + ti] = p;
    int rc = derive_cells(c);
    if (rc) {
        c->pairs[ti * c->ntypes + tj] = old_a;
        c->pairs[tj * c->ntypes + ti] = old_b;
        derive_cells(c);
        return rc;
    }
    c->table_dirty = true;
    if (c->ws_bound) {
        size_t need = workspace_bytes(c);
        if (need > c->ws_bytes) {
            c->ws_bound = false;
            c->state_set = false;
            return fail(c, SWP_ERR_STATE, "cell grid grew: workspace too small, bind a larger one");
        }
        refresh_layout(c);
        SWP_CUDA(c, cudaMemcpyAsync((void*)(c->precision == SWP_FP64 ? c->dd.cell_rank : c->df.cell_rank),
                                    c->cell_rank.data(), sizeof(int) * 2 * c->ncell,
                                    cudaMemcpyHostToDevice, c->stream));
    }
    return mark_stale(c);
}

int swp_set_bonds(swp_ctx* c, int n_bonds, const int32_t* bonds, double k, double r0)
{
    if (!c) return SWP_ERR_INVALID;
    if (n_bonds < 0 || (n_bonds > 0 && !bonds) || !(k >= 0.0) || !std::isfinite(k) || !(r0 >= 0.0) ||
        !std::isfinite(r0))
        return fail(c, SWP_ERR_INVALID, "need n_bonds >= 0, bonds, k >= 0, r0 >= 0");
    std::vector<int> tab;
    if (n_bonds > 0) {
        tab.assign((size_t)c->n * kMaxBonds, -1);
        std::vector<int> cnt(c->n, 0);
        for (int b = 0; b < n_bonds; b++) {
            const int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (i < 0 || j < 0 || i >= c->n || j >= c->n || i == j)
                return fail(c, SWP_ERR_INVALID, "bond with a tag out of range or bonded to itself");
            if (cnt[i] >= kMaxBonds || cnt[j] >= kMaxBonds)
                return fail(c, SWP_ERR_INVALID, "more than 4 bonds on one particle");
            for (int q = 0; q < cnt[i]; q++)
                if (tab[(size_t)i * kMaxBonds + q] == j) return fail(c, SWP_ERR_INVALID, "bond listed twice");
            tab[(size_t)i * kMaxBonds + cnt[i]++] = j;
            tab[(size_t)j * kMaxBonds + cnt[j]++] = i;
        }
    }
    c->bond_host.swap(tab);
    c->bond_k = k;
    c->bond_r0 = r0;
    c->bonds_dirty = !c->bond_host.empty();
    return mark_stale(c);
}

int swp_set_nlist(swp_ctx* c, double skin, int max_nn)
{
    if (!c) return SWP_ERR_INVALID;
    if (!(skin >= 0.0) || !std::isfinite(skin) || max_nn < 1 || max_nn > 4096)
        return fail(c, SWP_ERR_INVALID, "need skin >= 0 and 1 <= max_nn <= 4096");
    double old_skin = c->skin;
    int old_nn = c->max_nn;
    c->skin = skin;
    c->max_nn = max_nn;
    int rc = derive_cells(c);
    if (rc) {
        c->skin = old_skin;
        c->max_nn = old_nn;
        derive_cells(c);
        return rc;
    }
    c->table_dirty = true;
    if (max_nn != old_nn) c->nl_bound = false;
    if (c->ws_bound) {
        size_t need = workspace_bytes(c);
        if (need > c->ws_bytes) {
            c->ws_bound = false;
            c->state_set = false;
            return fail(c, SWP_ERR_STATE, "cell grid grew: workspace too small, bind a larger one");
        }
        refresh_layout(c);
        SWP_CUDA(c, cudaMemcpyAsync((void*)(c->precision == SWP_FP64 ? c->dd.cell_rank : c->df.cell_rank),
                                    c->cell_rank.data(), sizeof(int) * 2 * c->ncell,
                                    cudaMemcpyHostToDevice, c->stream));
    }
    return mark_stale(c);
}

int swp_workspace_size(const swp_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return SWP_ERR_INVALID;
    *bytes = workspace_bytes(const_cast<swp_ctx*>(c));
    return SWP_OK;
}

int swp_nlist_size(const swp_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return SWP_ERR_INVALID;
    *bytes = list_bytes(c);
    return SWP_OK;
}

int swp_bind_workspace(swp_ctx* c, void* ptr, size_t bytes, void* stream)
{
    if (!c) return SWP_ERR_INVALID;
    if (!ptr || ((uintptr_t)ptr & 255)) return fail(c, SWP_ERR_INVALID, "workspace must be 256-byte aligned");
    if (bytes < workspace_bytes(c)) return fail(c, SWP_ERR_INVALID, "workspace too small");
    c->ws = ptr;
    c->ws_bytes = bytes;
    c->stream = (cudaStream_t)stream;
    c->ws_bound = true;
    c->state_set = false;
    c->table_dirty = true;
    refresh_layout(c);
    SWP_CUDA(c, cudaMemcpyAsync((void*)(c->precision == SWP_FP64 ? c->dd.cell_rank : c->df.cell_rank),
                                c->cell_rank.data(), sizeof(int) * 2 * c->ncell, cudaMemcpyHostToDevice,
                                c->stream));
    return upload_table(c);
}

int swp_bind_nlist(swp_ctx* c, void* ptr, size_t bytes)
{
    if (!c) return SWP_ERR_INVALID;
    size_t need = 0;
    swp_nlist_size(c, &need);
    if (!ptr || ((uintptr_t)ptr & 255)) return fail(c, SWP_ERR_INVALID, "list buffer must be 256-byte aligned");
    if (bytes < need) return fail(c, SWP_ERR_INVALID, "neighbour-list buffer too small");
    c->nl = ptr;
    c->nl_bytes = bytes;
    c->nl_bound = true;
    if (c->ws_bound) refresh_layout(c);
    return mark_stale(c);
}

int swp_set_state(swp_ctx* c, const double* x, const double* v, const int32_t* type,
                  const double* mass, const int32_t* img, int where)
{
    int rc = ready(c, false);
    if (rc) return rc;
    if (where != SWP_HOST && where != SWP_DEVICE) return fail(c, SWP_ERR_INVALID, "bad where");
    const size_t n = (size_t)c->n;
    if (n > 0 && !x) return fail(c, SWP_ERR_INVALID, "positions required");
    if (where == SWP_HOST && n > 0) {
        for (size_t i = 0; i < 3 * n; i++)
            if (!std::isfinite(x[i]) || (v && !std::isfinite(v[i])))
                return fail(c, SWP_ERR_INVALID, "non-finite position or velocity");
        if (type)
            for (size_t i = 0; i < n; i++)
                if (type[i] < 0 || type[i] >= c->ntypes) return fail(c, SWP_ERR_INVALID, "type out of range");
        if (mass)
            for (size_t i = 0; i < n; i++)
                if (!(mass[i] > 0.0) || !std::isfinite(mass[i])) return fail(c, SWP_ERR_INVALID, "mass must be > 0");
    }
    rc = upload_table(c);
    if (rc) return rc;
    double* io;
    int* io_int;
    Ctl* ctl;
    if (c->precision == SWP_FP64) {
        io = c->dd.io;
        io_int = c->dd.io_int;
        ctl = c->dd.ctl;
    } else {
        io = c->df.io;
        io_int = c->df.io_int;
        ctl = c->df.ctl;
    }
    std::memset(&c->hctl, 0, sizeof(Ctl));
    c->hctl.state = 1;
    c->hctl.need_rebuild = 1;
    SWP_CUDA(c, cudaMemcpyAsync(ctl, &c->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    // the cell build expects zeroed counts (it zeroes them itself after use)
    SWP_CUDA(c, cudaMemsetAsync(c->precision == SWP_FP64 ? (void*)c->dd.cell_cnt : (void*)c->df.cell_cnt, 0,
                                sizeof(int) * c->ncell, c->stream));
    if (n == 0) {
        c->state_set = true;
        return SWP_OK;
    }
    SWP_CUDA(c, cudaMemcpyAsync(io, x, sizeof(double) * 3 * n, kind_to_dev(where), c->stream));
    if (v) SWP_CUDA(c, cudaMemcpyAsync(io + 3 * n, v, sizeof(double) * 3 * n, kind_to_dev(where), c->stream));
    else SWP_CUDA(c, cudaMemsetAsync(io + 3 * n, 0, sizeof(double) * 3 * n, c->stream));
    if (mass) SWP_CUDA(c, cudaMemcpyAsync(io + 6 * n, mass, sizeof(double) * n, kind_to_dev(where), c->stream));
    else {
        std::vector<double> ones(n, 1.0);
        SWP_CUDA(c, cudaMemcpyAsync(io + 6 * n, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (type) SWP_CUDA(c, cudaMemcpyAsync(io_int, type, sizeof(int) * n, kind_to_dev(where), c->stream));
    else SWP_CUDA(c, cudaMemsetAsync(io_int, 0, sizeof(int) * n, c->stream));
    if (img) SWP_CUDA(c, cudaMemcpyAsync(io_int + n, img, sizeof(int) * 3 * n, kind_to_dev(where), c->stream));
    else SWP_CUDA(c, cudaMemsetAsync(io_int + n, 0, sizeof(int) * 3 * n, c->stream));
    if (c->precision == SWP_FP64) SWP_CUDA(c, launch_set_state<double>(c->dd, c->stream));
    else SWP_CUDA(c, launch_set_state<float>(c->df, c->stream));
    c->state_set = true;
    return SWP_OK;
}

int swp_set_step(swp_ctx* c, int64_t step)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (step < 0) return fail(c, SWP_ERR_INVALID, "step must be >= 0");
    if (c->n == 0) return SWP_OK;
    static_assert(sizeof(long long) == sizeof(int64_t), "step width");
    long long s = (long long)step;
    SWP_CUDA(c, cudaMemcpyAsync(&dev_ctl(c)->step, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
    SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    return SWP_OK;
}

int swp_build_nlist(swp_ctx* c)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (c->n == 0) return SWP_OK;
    RunArgs a;
    std::memset(&a, 0, sizeof(a));
    a.build_only = 1;
    return run_any(c, a);
}

int swp_compute_forces(swp_ctx* c)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (c->n == 0) return SWP_OK;
    RunArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nsteps = 0;
    return run_any(c, a);
}

static bool step_params_ok(double dt, double kT, double gamma, int nsteps)
{
    return dt > 0.0 && std::isfinite(dt) && nsteps >= 0 && gamma >= 0.0 && kT >= 0.0 &&
           std::isfinite(gamma) && std::isfinite(kT);
}

// Integrator constants of a run (BAOAB when gamma > 0, else velocity Verlet).
static RunArgs step_args(double dt, double kT, double gamma, int nsteps)
{
    RunArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nsteps = nsteps;
    a.dt = dt;
    a.langevin = gamma > 0.0 ? 1 : 0;
    a.c1 = std::exp(-gamma * dt);
    a.c2 = std::sqrt((1.0 - a.c1 * a.c1) * kT);
    a.hdt_d = 0.5 * dt;
    a.c1_d = a.c1;
    a.c2_d = a.c2;
    a.hdt_f = (float)a.hdt_d;
    a.c1_f = (float)a.c1;
    a.c2_f = (float)a.c2;
    return a;
}

static int step_common(swp_ctx* c, double dt, double kT, double gamma, int nsteps)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (!step_params_ok(dt, kT, gamma, nsteps))
        return fail(c, SWP_ERR_INVALID, "need dt > 0, nsteps >= 0, gamma >= 0, kT >= 0");
    if (c->n == 0 || nsteps == 0) return SWP_OK;
    return run_any(c, step_args(dt, kT, gamma, nsteps));
}

int swp_step_nve(swp_ctx* c, double dt, int nsteps) { return step_common(c, dt, 0.0, 0.0, nsteps); }

int swp_step_nvt(swp_ctx* c, double dt, double kT, double gamma, int nsteps)
{
    return step_common(c, dt, kT, gamma, nsteps);
}

size_t swp_batch_workspace_size(int n_systems)
{
    if (n_systems < 1) return 0;
    return batch_bytes(n_systems, std::max(sizeof(Dev<float>), sizeof(Dev<double>)));
}

int swp_batch_step(swp_ctx* const* ctx, int n_systems, const double* dt, const double* kT,
                   const double* gamma, int nsteps, double split, int threads, void* ws, size_t ws_bytes)
{
    if (!ctx || n_systems < 1 || !dt || !kT || !gamma || !ws || nsteps < 0 || !(split >= 0.0))
        return SWP_ERR_INVALID;
    if (threads == 0) threads = 1024;
    for (int r = 0; r < n_systems; r++)
        if (!ctx[r]) return SWP_ERR_INVALID;
    swp_ctx* c0 = ctx[0];
    std::vector<int> idx;
    std::vector<RunArgs> args;
    for (int r = 0; r < n_systems; r++) {
        swp_ctx* c = ctx[r];
        int rc = ready(c, true);
        if (rc) return rc;
        if (c->precision != c0->precision || c->device != c0->device || c->stream != c0->stream)
            return fail(c0, SWP_ERR_INVALID, "batched systems need one precision, device and stream");
        if (!batch_shape_ok(c->precision, threads))
            return fail(c0, SWP_ERR_INVALID, "block shape: 1024 threads, or 512, 384 or 256 in FP32");
        if (!step_params_ok(dt[r], kT[r], gamma[r], nsteps))
            return fail(c, SWP_ERR_INVALID, "need dt > 0, nsteps >= 0, gamma >= 0, kT >= 0");
        for (int q = 0; q < r; q++)
            if (ctx[q] == c) return fail(c0, SWP_ERR_INVALID, "a system appears twice in the batch");
        if (c->n == 0) continue;
        idx.push_back(r);
        args.push_back(step_args(dt[r], kT[r], gamma[r], nsteps));
    }
    if (idx.empty() || nsteps == 0) return SWP_OK;
    return c0->precision == SWP_FP64 ? batch_run<double>(ctx, idx, args, split, threads, ws, ws_bytes)
                                     : batch_run<float>(ctx, idx, args, split, threads, ws, ws_bytes);
}

int swp_batch_plan(const long long* w, int n_systems, int n_blocks, double split, int max_group, int min_part,
                   int* item_ofs, int* items, int* n_items)
{
    if (!w || n_systems < 1 || n_blocks < 1 || n_blocks > kMaxGrid || !(split >= 0.0) || max_group < 1 ||
        min_part < 1 || !item_ofs || !items || !n_items)
        return SWP_ERR_INVALID;
    std::vector<long long> wv(w, w + n_systems);
    for (long long x : wv)
        if (x < 0) return SWP_ERR_INVALID;
    BatchPlan plan;
    if (plan_batch(wv, n_blocks, split, max_group, min_part, plan)) return SWP_ERR_INVALID;
    if (plan.items.size() > (size_t)n_systems + n_blocks) return SWP_ERR_INVALID;
    for (int k = 0; k <= n_blocks; k++) item_ofs[k] = plan.item_ofs[k];
    for (size_t i = 0; i < plan.items.size(); i++) {
        items[4 * i + 0] = plan.items[i].x;
        items[4 * i + 1] = plan.items[i].y;
        items[4 * i + 2] = plan.items[i].z;
        items[4 * i + 3] = plan.items[i].w;
    }
    *n_items = (int)plan.items.size();
    return SWP_OK;
}

int swp_sync(swp_ctx* c)
{
    if (!c) return SWP_ERR_INVALID;
    if (!c->ws_bound) return SWP_OK;
    return sync_ctl(c);
}

int swp_read_thermo(swp_ctx* c, swp_thermo* out)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (!out) return fail(c, SWP_ERR_INVALID, "null output");
    rc = sync_ctl(c);
    std::memset(out, 0, sizeof(*out));
    const Ctl& h = c->hctl;
    out->U2 = h.thermo[Q_U2];
    out->U3 = h.thermo[Q_U3];
    out->K = h.thermo[Q_K];
    for (int k = 0; k < 6; k++) out->W[k] = h.thermo[Q_W0 + k];
    out->n_bonds = (int64_t)std::llround(h.thermo[Q_BONDS]);
    out->step = h.step;
    out->n_rebuilds = h.n_rebuilds;
    out->steps_done = h.steps_done;
    out->max_row = h.max_row;
    out->state = h.state;
    out->resident_steps = h.resident_steps;
    return rc;
}

int swp_read_forces(swp_ctx* c, double* f, int where)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (c->n == 0) return SWP_OK;
    if (!f) return fail(c, SWP_ERR_INVALID, "null output");
    rc = sync_ctl(c);
    if (rc) return rc;
    if (c->hctl.state != 0) return fail(c, SWP_ERR_STATE, "forces are not current: call swp_compute_forces");
    double* io;
    if (c->precision == SWP_FP64) {
        SWP_CUDA(c, launch_get_forces<double>(c->dd, c->hctl.pos_cur, c->stream));
        io = c->dd.io;
    } else {
        SWP_CUDA(c, launch_get_forces<float>(c->df, c->hctl.pos_cur, c->stream));
        io = c->df.io;
    }
    SWP_CUDA(c, cudaMemcpyAsync(f, io, sizeof(double) * 3 * c->n, kind_from_dev(where), c->stream));
    SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    return SWP_OK;
}

int swp_param_grad(swp_ctx* c, int ti, int tj, double dU[3], double* dF_dev)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (!dU) return fail(c, SWP_ERR_INVALID, "null output");
    if (ti < 0 || tj < 0 || ti >= c->ntypes || tj >= c->ntypes) return fail(c, SWP_ERR_INVALID, "type out of range");
    const PairHost& p = c->pairs[ti * c->ntypes + tj];
    if (p.kind != KIND_SWAP) return fail(c, SWP_ERR_INVALID, "(ti, tj) is not a swap pair");
    if (p.shift) return fail(c, SWP_ERR_INVALID, "parameter derivatives need the unshifted form");
    for (int a = 0; a < c->ntypes; a++)
        for (int b = a; b < c->ntypes; b++)
            if (c->pairs[a * c->ntypes + b].kind == KIND_SWAP && !((a == ti && b == tj) || (a == tj && b == ti)))
                return fail(c, SWP_ERR_INVALID, "parameter derivatives need a single reactive type pair");
    dU[0] = dU[1] = dU[2] = 0.0;
    if (c->n == 0) return SWP_OK;
    rc = sync_ctl(c);
    if (rc) return rc;
    if (c->hctl.state != 0) return fail(c, SWP_ERR_STATE, "forces are not current: call swp_compute_forces");
    // theta and dU/dtheta pass through the scratch after the four sums
    double th[3] = {p.lambda3, p.eps, p.sigma}, out[3];
    double* part = c->precision == SWP_FP64 ? c->dd.partials : c->df.partials;
    double* dth = part + 2048 + 4;
    double* ddu = dth + 3;
    SWP_CUDA(c, cudaMemcpyAsync(dth, th, sizeof th, cudaMemcpyHostToDevice, c->stream));
    if (c->precision == SWP_FP64)
        SWP_CUDA(c, launch_param_grad<double>(c->dd, c->hctl.pos_cur, c->dd.io, part, dth, dF_dev, part + 2048,
                                               ddu, c->stream));
    else
        SWP_CUDA(c, launch_param_grad<float>(c->df, c->hctl.pos_cur, c->df.io, part, dth, dF_dev, part + 2048,
                                              ddu, c->stream));
    SWP_CUDA(c, cudaMemcpyAsync(out, ddu, sizeof out, cudaMemcpyDeviceToHost, c->stream));
    SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    dU[0] = out[0];
    dU[1] = out[1];
    dU[2] = out[2];
    return SWP_OK;
}

int swp_eval_grad(swp_ctx* c, int ti, int tj, const double* theta_dev, const double* x_dev, const int32_t* type_dev,
                  double* U_dev, double* F_dev, double* dU_dev, double* dF_dev)
{
    int rc = ready(c, false);
    if (rc) return rc;
    if (!theta_dev || !U_dev || (c->n > 0 && !x_dev)) return fail(c, SWP_ERR_INVALID, "null theta, x or U");
    if (ti < 0 || tj < 0 || ti >= c->ntypes || tj >= c->ntypes) return fail(c, SWP_ERR_INVALID, "type out of range");
    const PairHost& p = c->pairs[ti * c->ntypes + tj];
    if (p.kind != KIND_SWAP) return fail(c, SWP_ERR_INVALID, "(ti, tj) is not a swap pair");
    if (p.shift) return fail(c, SWP_ERR_INVALID, "parameter derivatives need the unshifted form");
    for (int a = 0; a < c->ntypes; a++)
        for (int b = a; b < c->ntypes; b++)
            if (c->pairs[a * c->ntypes + b].kind == KIND_SWAP && !((a == ti && b == tj) || (a == tj && b == ti)))
                return fail(c, SWP_ERR_INVALID, "parameter derivatives need a single reactive type pair");
    rc = upload_table(c);
    if (rc) return rc;
    const size_t n = (size_t)c->n;
    const double c_rmin = std::pow(2.0, 1.0 / p.n), c_rb = std::pow((1.0 - std::sqrt(0.5)) / 2.0, -1.0 / p.n);
    const bool f64 = c->precision == SWP_FP64;
    double* io = f64 ? c->dd.io : c->df.io;
    SWP_CUDA(c, cudaMemsetAsync(f64 ? (void*)c->dd.cell_cnt : (void*)c->df.cell_cnt, 0, sizeof(int) * c->ncell,
                                c->stream));
    if (n > 0) SWP_CUDA(c, cudaMemcpyAsync(io, x_dev, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, c->stream));
    if (f64) SWP_CUDA(c, launch_eval_prep<double>(c->dd, ti, tj, theta_dev, c_rmin, c_rb, p.rbond, type_dev, c->stream));
    else SWP_CUDA(c, launch_eval_prep<float>(c->df, ti, tj, theta_dev, c_rmin, c_rb, p.rbond, type_dev, c->stream));
    c->state_set = true;
    c->table_theta = true;
    if (n == 0) {
        SWP_CUDA(c, cudaMemsetAsync(U_dev, 0, sizeof(double), c->stream));
        if (dU_dev) SWP_CUDA(c, cudaMemsetAsync(dU_dev, 0, 3 * sizeof(double), c->stream));
        return SWP_OK;
    }
    if (f64) SWP_CUDA(c, launch_set_state<double>(c->dd, c->stream));
    else SWP_CUDA(c, launch_set_state<float>(c->df, c->stream));
    // forces at the new positions: rebuild and evaluate, coefficients from the device table
    RunArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nsteps = 0;
    a.force_rebuild = 1;
    c->table_only = 1;
    rc = run_any(c, a);
    c->table_only = 0;
    if (rc) return rc;
    k_eval_energy<<<1, 1, 0, c->stream>>>(dev_ctl(c), U_dev);
    SWP_CUDA(c, cudaGetLastError());
    if (F_dev) {
        if (f64) SWP_CUDA(c, launch_get_forces<double>(c->dd, -1, c->stream));
        else SWP_CUDA(c, launch_get_forces<float>(c->df, -1, c->stream));
        SWP_CUDA(c, cudaMemcpyAsync(F_dev, io, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (dU_dev || dF_dev) {
        double* part = f64 ? c->dd.partials : c->df.partials;
        if (f64)
            SWP_CUDA(c, launch_param_grad<double>(c->dd, -1, io, part, theta_dev, dF_dev, part + 2048, dU_dev, c->stream));
        else
            SWP_CUDA(c, launch_param_grad<float>(c->df, -1, io, part, theta_dev, dF_dev, part + 2048, dU_dev, c->stream));
    }
    return SWP_OK;
}

int swp_read_state(swp_ctx* c, double* x, double* v, int32_t* img, int where)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (c->n == 0) return SWP_OK;
    rc = sync_ctl(c);
    if (rc && rc != SWP_ERR_NLIST_OVERFLOW) return rc;
    const size_t n = (size_t)c->n;
    double* io;
    int* io_int;
    if (c->precision == SWP_FP64) {
        SWP_CUDA(c, launch_get_state<double>(c->dd, c->hctl.pos_cur, c->hctl.arr_cur, c->stream));
        io = c->dd.io;
        io_int = c->dd.io_int;
    } else {
        SWP_CUDA(c, launch_get_state<float>(c->df, c->hctl.pos_cur, c->hctl.arr_cur, c->stream));
        io = c->df.io;
        io_int = c->df.io_int;
    }
    if (x) SWP_CUDA(c, cudaMemcpyAsync(x, io, sizeof(double) * 3 * n, kind_from_dev(where), c->stream));
    if (v) SWP_CUDA(c, cudaMemcpyAsync(v, io + 3 * n, sizeof(double) * 3 * n, kind_from_dev(where), c->stream));
    if (img) SWP_CUDA(c, cudaMemcpyAsync(img, io_int + n, sizeof(int) * 3 * n, kind_from_dev(where), c->stream));
    SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    return rc;
}

int swp_read_nlist(swp_ctx* c, int32_t* rows_dev, int32_t* counts_dev, int width)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (c->n == 0) return SWP_OK;
    if (!rows_dev || !counts_dev || width < 1) return fail(c, SWP_ERR_INVALID, "null output or width < 1");
    rc = sync_ctl(c);
    if (rc) return rc;
    if (c->hctl.need_rebuild) return fail(c, SWP_ERR_STATE, "neighbour list is stale: call swp_build_nlist");
    if (c->precision == SWP_FP64) SWP_CUDA(c, launch_get_nlist<double>(c->dd, c->hctl.pos_cur, rows_dev, counts_dev, width, c->stream));
    else SWP_CUDA(c, launch_get_nlist<float>(c->df, c->hctl.pos_cur, rows_dev, counts_dev, width, c->stream));
    SWP_CUDA(c, cudaStreamSynchronize(c->stream));
    return SWP_OK;
}

int swp_set_launch(swp_ctx* c, int blocks_per_sm)
{
    if (!c) return SWP_ERR_INVALID;
    if (blocks_per_sm < 0) return fail(c, SWP_ERR_INVALID, "blocks_per_sm must be >= 0");
    c->bps_req = blocks_per_sm;
    if (c->ws_bound && c->state_set && c->n > 0) return mark_stale(c);
    return SWP_OK;
}

int swp_set_grid(swp_ctx* c, int blocks)
{
    if (!c) return SWP_ERR_INVALID;
    if (blocks < 0) return fail(c, SWP_ERR_INVALID, "blocks must be >= 0");
    c->grid_req = blocks;
    if (c->ws_bound && c->state_set && c->n > 0) return mark_stale(c);
    return SWP_OK;
}

int swp_set_timeout(swp_ctx* c, int64_t ns)
{
    if (!c) return SWP_ERR_INVALID;
    if (ns < 1000) return fail(c, SWP_ERR_INVALID, "timeout must be >= 1000 ns");
    c->timeout_ns = (long long)ns;
    return SWP_OK;
}

int swp_set_resident(swp_ctx* c, int enable)
{
    if (!c) return SWP_ERR_INVALID;
    if (enable != 0 && enable != 1) return fail(c, SWP_ERR_INVALID, "enable must be 0 or 1");
    c->resident = enable;
    return SWP_OK;
}

size_t swp_thermo_log_bytes(const swp_ctx* c, int64_t capacity)
{
    if (!c || capacity < 1 || capacity > INT32_MAX || c->max_blocks < 1) return 0;
    return ((sizeof(double) * (size_t)capacity * c->max_blocks * kNQ + 255) & ~(size_t)255) +
           sizeof(long long) * 2 * (size_t)capacity;
}

int swp_set_thermo_log(swp_ctx* c, int every, int64_t capacity, void* ring, size_t ring_bytes)
{
    if (!c) return SWP_ERR_INVALID;
    if (every < 0) return fail(c, SWP_ERR_INVALID, "every must be >= 0");
    if (every > 0) {
        const size_t need = swp_thermo_log_bytes(c, capacity);
        if (need == 0) return fail(c, SWP_ERR_INVALID, "capacity must be in [1, 2^31 - 1]");
        if (!ring || ((uintptr_t)ring & 255)) return fail(c, SWP_ERR_INVALID, "ring must be a 256-byte aligned device buffer");
        if (ring_bytes < need) return fail(c, SWP_ERR_INVALID, "ring smaller than swp_thermo_log_bytes");
    }
    double* rec = every > 0 ? (double*)ring : nullptr;
    long long* stp = every > 0 ? (long long*)((char*)ring + ((sizeof(double) * (size_t)capacity * c->max_blocks * kNQ + 255) &
                                                            ~(size_t)255))
                               : nullptr;
    const int cap = every > 0 ? (int)capacity : 0;
    c->df.tlog = c->dd.tlog = rec;
    c->df.tlog_step = c->dd.tlog_step = stp;
    c->df.tlog_cap = c->dd.tlog_cap = cap;
    c->tlog_every = every;
    if (c->ws_bound) {
        SWP_CUDA(c, cudaMemsetAsync(&dev_ctl(c)->tlog_n, 0, sizeof(long long), c->stream));
    }
    return SWP_OK;
}

int swp_thermo_log(swp_ctx* c, double* rec_dev, int64_t* step_dev, int64_t max_records, int64_t* n_records)
{
    int rc = ready(c, true);
    if (rc) return rc;
    if (!n_records || max_records < 0) return fail(c, SWP_ERR_INVALID, "need n_records and max_records >= 0");
    *n_records = 0;
    if (!c->df.tlog) return fail(c, SWP_ERR_INVALID, "no thermo log set (swp_set_thermo_log)");
    if (max_records > 0 && (!rec_dev || !step_dev)) return fail(c, SWP_ERR_INVALID, "null output buffer");
    rc = sync_ctl(c);
    if (rc) return rc;
    const long long written = c->hctl.tlog_n;
    const long long n = std::min<long long>(std::min<long long>(written, c->df.tlog_cap), max_records);
    if (n <= 0) return SWP_OK;
    k_tlog_reduce<<<(unsigned)n, 32 * kNQA, 0, c->stream>>>(c->df.tlog, c->df.tlog_step, c->df.tlog_cap,
                                                             c->max_blocks, written - n, rec_dev,
                                                             (long long*)step_dev);
    SWP_CUDA(c, cudaGetLastError());
    *n_records = n;
    return SWP_OK;
}

int swp_set_withhold_arrival(swp_ctx* c, int on)
{
    if (!c) return SWP_ERR_INVALID;
    if (on != 0 && on != 1) return fail(c, SWP_ERR_INVALID, "on must be 0 or 1");
    c->withhold = on;
    return SWP_OK;
}

const char* swp_last_error(const swp_ctx* c) { return c ? c->err.c_str() : "null context"; }

int swp_destroy(swp_ctx* c)
{
    delete c;
    return SWP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Force evaluation without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need forces:
// code embedded in a host framework whose memory pool has reserved the
// device's memory and forbids side allocations, or a latency-bound loop that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.
// swp_compute_forces_static serves them: its scratch (state copy, cell list,
// neighbour list, partial sums) lives in the fixed-size array below, which the
// library's module reserves on every GPU that loads it, for the life of the
// process.  The call synchronises its stream and uploads small parameter
// blocks from pageable host memory, so it is not for stream capture.

namespace {

constexpr size_t kStaticScratchBytes = (size_t)SWP_STATIC_SCRATCH_BYTES;
constexpr int kMaxStaticDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device (host code sees only a
// stand-in symbol; the address comes from cudaGetSymbolAddress).
static void* g_static_addr[kMaxStaticDevices];

__global__ void k_static_stage(const double* x, const int32_t* type, double* io, int* io_int, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; c++) {
            io[3 * i + c] = x[3 * i + c];
            io[3 * n + 3 * i + c] = 0.0;  // velocities
            io_int[n + 3 * i + c] = 0;    // images
        }
        io[6 * n + i] = 1.0;  // masses
        io_int[i] = type ? type[i] : 0;
    }
}

template <typename Real>
int static_forces(swp_ctx* c, const double* x, const int32_t* type, double* f, double* thermo,
                  cudaStream_t s)
{
    int dev = 0;
    SWP_CUDA(c, cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(c, SWP_ERR_INVALID, "the current device is not the one the context was created on");
    if (dev < 0 || dev >= kMaxStaticDevices) return fail(c, SWP_ERR_INVALID, "device index too large");
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        SWP_CUDA(c, cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_addr[dev] = p;
    }
    if (!c->bond_host.empty()) return fail(c, SWP_ERR_INVALID, "bonded systems are not supported here");
    char* base = (char*)g_static_addr[dev];
    const size_t ws = layout<Real>(c, nullptr, nullptr);
    const size_t nl = list_bytes(c);
    if (ws + nl > kStaticScratchBytes) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "system needs %zu bytes of scratch; the static scratch holds %zu "
                      "(fewer particles, a smaller max_nn or a denser box fit)",
                      ws + nl, kStaticScratchBytes);
        return fail(c, SWP_ERR_INVALID, buf);
    }
    Dev<Real> d{};
    layout<Real>(c, base, &d);
    set_list(c, base + ws, &d);

    PairP<Real> tab[kMaxTypes * kMaxTypes];
    fill_pair_table<Real>(c, tab);
    SWP_CUDA(c, cudaMemcpyAsync((void*)d.table, tab, sizeof(tab), cudaMemcpyHostToDevice, s));
    SWP_CUDA(c, cudaMemcpyAsync((void*)d.cell_rank, c->cell_rank.data(), sizeof(int) * 2 * c->ncell,
                                cudaMemcpyHostToDevice, s));
    // The array keeps the previous call's contents: the control block (status,
    // barrier counter, state) must start from zero every call.
    Ctl h;
    std::memset(&h, 0, sizeof(h));
    h.state = 1;
    h.need_rebuild = 1;
    SWP_CUDA(c, cudaMemcpyAsync(d.ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    SWP_CUDA(c, cudaMemsetAsync(d.cell_cnt, 0, sizeof(int) * c->ncell, s));
    k_static_stage<<<(c->n + 255) / 256, 256, 0, s>>>(x, type, d.io, d.io_int, c->n);
    SWP_CUDA(c, cudaGetLastError());
    SWP_CUDA(c, launch_set_state<Real>(d, s));

    int bps = 0;
    SWP_CUDA(c, run_occupancy<Real>(kBlock, &bps));
    if (bps < 1) return fail(c, SWP_ERR_CUDA, "step kernel does not fit on an SM");
    if (c->bps_req > 0) bps = std::min(bps, c->bps_req);
    bps = std::min(bps, c->max_blocks / std::max(c->num_sms, 1));
    RunArgs a;
    std::memset(&a, 0, sizeof(a));
    a.max_blocks = c->max_blocks;
    a.timeout_ns = c->timeout_ns;
    a.skin_eff = c->skin;
    a.seed = c->seed;
    SWP_CUDA(c, launch_run<Real>(d, a, step_grid(c, bps), kBlock, s));
    SWP_CUDA(c, cudaMemcpyAsync(&h, d.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
    SWP_CUDA(c, cudaStreamSynchronize(s));
    if (h.status & kStatusTimeout) return fail(c, SWP_ERR_TIMEOUT, "a device-side wait timed out");
    if (h.status & kStatusNonfinite) return fail(c, SWP_ERR_NONFINITE, "non-finite force");
    if (h.status & kStatusOverflow) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "neighbour row of %d entries exceeds max_nn = %d", h.max_row,
                      c->max_nn);
        return fail(c, SWP_ERR_NLIST_OVERFLOW, buf);
    }
    SWP_CUDA(c, launch_get_forces<Real>(d, h.pos_cur, s));
    SWP_CUDA(c, cudaMemcpyAsync(f, d.io, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, s));
    if (thermo) {
        // [U2, U3, W xx yy zz xy xz yz, n_bonds]
        SWP_CUDA(c, cudaMemcpyAsync(thermo, &d.ctl->thermo[Q_U2], 2 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        SWP_CUDA(c, cudaMemcpyAsync(thermo + 2, &d.ctl->thermo[Q_W0], 7 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
    }
    SWP_CUDA(c, cudaStreamSynchronize(s));
    return SWP_OK;
}

}  // namespace

extern "C" int swp_compute_forces_static(swp_ctx* c, const double* x_dev, const int32_t* type_dev,
                                         double* f_dev, double* thermo_dev, void* cuda_stream)
{
    if (!c) return SWP_ERR_INVALID;
    if (c->n == 0) return SWP_OK;
    if (!x_dev || !f_dev) return fail(c, SWP_ERR_INVALID, "positions and forces are required");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    return c->precision == SWP_FP64 ? static_forces<double>(c, x_dev, type_dev, f_dev, thermo_dev, s)
                                    : static_forces<float>(c, x_dev, type_dev, f_dev, thermo_dev, s);
}
