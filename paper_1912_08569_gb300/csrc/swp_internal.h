// Internal layout shared by the CUDA kernels and the host side of the C-ABI.
// Not part of the public interface (that is include/swapmd.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace swp {

constexpr int kMaxTypes = 8;       // type-pair table is kMaxTypes^2 entries at most
constexpr int kNQ = 12;            // per-block thermo partials: see Q_* below
constexpr int kTypeBits = 4;       // packed word: (tag << kTypeBits) | type
constexpr int kBlock = 768;        // threads per block of the step kernel (one block per SM, 80 registers)
constexpr int kMaxGrid = 320;      // largest grid of the step kernel (blocks)
constexpr int kBlockBatch = 1024;  // threads per block of the batched kernel
constexpr int kBlockWide = 1024;   // threads per block of the step kernel of bonded networks
constexpr int kMaxBonds = 4;       // harmonic bonds per particle (chains: 2)
constexpr int kMaxTag = (1 << 27); // tags must fit in 27 bits (sign bit stays clear)

// Thermo quantities, in the order of the per-block partials.
enum { Q_U2 = 0, Q_U3 = 1, Q_K = 2, Q_W0 = 3, Q_BONDS = 9, Q_SPARE0 = 10, Q_SPARE1 = 11 };
constexpr int kNQA = 10;  // quantities accumulated per thread (Q_U2 .. Q_BONDS)

// Fixed-point position unit: positions are int64 multiples of 2^-48 sigma.
constexpr double kFix = 281474976710656.0;          // 2^48
constexpr double kInvFix = 3.5527136788005009e-15;  // 2^-48

enum PairKind { KIND_NONE = 0, KIND_WCA = 1, KIND_SWAP = 2 };

// One type-pair entry, precomputed on the host in double and stored in the
// arithmetic precision of the run.
template <typename Real>
struct PairP {
    int kind;   // PairKind
    int nhalf;  // exponent n = 2*nhalf + odd
    int odd;
    int pad;
    Real four_eps;    // 4 eps
    Real n_real;      // n
    Real sig2;        // sigma^2
    Real rc2;         // squared interaction cut-off (decision threshold)
    Real rmin2;       // squared r_min = (sigma 2^(1/n))^2
    Real a;           // sqrt(lambda eps): triplet prefactor factor
    Real inv_epshat;  // 1 / (eps + v(r_cut)) shifted, 1 / eps unshifted
    Real vshift;      // v(r_cut) shifted, 0 unshifted (vh = (vshift - v) inv_epshat)
    Real ushift;      // two-body energy offset: -vshift (swap), +eps (wca)
    Real rlist2;      // squared neighbour-list radius (decision threshold), < 0: never
    Real rbond2;      // squared bond radius (decision threshold)
};

// Device-side control block (one per context, in the workspace).
struct Ctl {
    unsigned long long barrier;  // grid-barrier arrival counter (zeroed before each launch)
    int status;                  // latched SWP_* error bits (see kStatus*)
    int state;                   // 0: full step, forces valid; 1: forces invalid; 2: mid-step
    int pos_cur;                 // which pos buffer holds the current snapshot
    int arr_cur;                 // which xq/img/vel buffer set is current
    int need_rebuild;            // set by the host after set_state / parameter changes
    int max_row;                 // row length (entries per particle) the last build needed
    int overflow;                // set by a block whose entries exceeded its capacity
    int list_grid;               // grid size the list was built for (its block partition)
    int list_chunk;              // block size the list was built with (its sub-chunk length)
    unsigned int dmax2[2];       // per-step max squared displacement (float bits), by parity
    double disp;                 // displacement bound accumulated since the last build
    long long step;              // completed time steps
    long long n_rebuilds;
    long long steps_done;        // steps completed by the last run call
    long long timeout_at;        // diagnostic: phase id where a wait gave up
    double thermo[kNQ];          // last reduced thermo record
    int rfail[2];                // resident-mode agreement: a block whose local structures do not
                                 // fit sets its round's word (rounds alternate; cleared on device)
    int resident_steps;          // steps of the last run call taken in the resident mode
    int pad_;
    long long tlog_n;            // thermo-log records written since the log was set
};

// Status bits latched on the device.
constexpr int kStatusOverflow = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusNonfinite = 4;
constexpr int kStatusBadCell = 8;
constexpr int kStatusBadType = 16;  // a state's type (device input) out of range

template <typename Real>
struct Vec4;
template <>
struct Vec4<float> {
    typedef float4 type;
};
struct alignas(32) dbl4 {
    double x, y, z, w;
};
template <>
struct Vec4<double> {
    typedef dbl4 type;
};

// Position snapshot of one particle: FP64, (x, y, z, packed bits) in double;
// FP32, (u, v, w, packed bits) with each coordinate a 32-bit fraction of its
// box edge (see Dev::fmul).
template <typename Real>
struct PosVec;
template <>
struct PosVec<float> {
    typedef int4 type;
};
template <>
struct PosVec<double> {
    typedef dbl4 type;
};

// Pointers and sizes of one context's device state (passed by value).
template <typename Real>
struct Dev {
    typedef typename Vec4<Real>::type R4;
    typedef typename PosVec<Real>::type P4;
    int n;
    int ntypes;
    int max_nn;
    int ncell;
    int nc[3];
    Real L[3];
    Real hL[3];
    Real inv_cw[3];  // cells per unit length
    Real iL[3];      // 1 / L
    long long Lq[3]; // box in fixed-point units
    // FP32 snapshot coordinates: u = floor(q fmul / 2^64) with q the fixed-point
    // coordinate and fmul = floor(2^96 / Lq), a 32-bit fraction of the box edge;
    // a displacement is the wrap-around difference of two fractions (the
    // minimum image) times fscale = Lq 2^-80, the box edge per 2^32
    unsigned long long fmul[3];
    float fscale[3];
    P4* pos[2];      // snapshot (coordinates, packed tag/type bits), ping-pong
    long long* xq[2];  // fixed-point positions, SoA [3][n], two sets (reorder)
    int* img[2];       // image counts, SoA [3][n], two sets
    R4* vel[2];        // (vx, vy, vz, 1/m), two sets
    R4* force;         // (fx, fy, fz, 0)
    Real* S;           // per-centre sum of a*vh over reactive partners
    int* ent_j;            // neighbour entries: partner slot (block-compact layout)
    unsigned short* ent_o; // neighbour entries: owner's index inside its sub-chunk (< 1024)
    int4* pinfo;           // per particle: (first reactive entry, count, first other entry, count)
    const int* cell_rank;  // [2 * ncell]: cell linear index -> rank in the sorted cell order,
                           // then rank -> linear index
    int* cell_cnt;     // [ncell]
    int* cell_start;   // [ncell + 1]
    int* cell_fill;    // [ncell]
    int* perm;         // [n] new slot -> old slot
    int* bsum;         // [max_blocks] per-block cell-count sums (scan)
    double* partials;  // [max_blocks][kNQ]
    Ctl* ctl;
    double* io;        // host-exchange staging: [3n] x, [3n] v, [n] mass
    int* io_int;       // staging: [n] types, [3n] images
    const PairP<Real>* table;  // [ntypes * ntypes]
    int* bond_tag;     // [n][kMaxBonds] bonded partners' tags by tag (-1: none)
    int* slot_of_tag;  // [n] slot of every tag (written at each rebuild when has_bonds)
    int has_bonds;     // harmonic bonds k/2 (r - r0)^2 act (the vitrimer network's chains)
    Real bond_k, bond_r0;
    // thermo log (null: none): a ring of tlog_cap records, each the block partials
    // [max_blocks][kNQ] of one logged step, with (step, grid size) in tlog_step[2 r]
    double* tlog;
    long long* tlog_step;
    int tlog_cap;
};

// What one launch of the step kernel does.
struct RunArgs {
    int nsteps;         // time steps to advance (0: only bring forces up to date)
    int build_only;     // 1: rebuild the neighbour list and stop
    int force_rebuild;  // 1: rebuild before the first force evaluation
    int langevin;       // 1: BAOAB with the O step; 0: velocity Verlet
    double dt;
    double c1;          // exp(-gamma dt)
    double c2;          // sqrt((1 - c1^2) kT)
    // the same in the arithmetic precision of the run (converted once on the host)
    float hdt_f, c1_f, c2_f;
    double hdt_d, c1_d, c2_d;
    double skin_eff;    // rebuild when 2 * displacement bound > skin_eff
    unsigned long long seed;
    long long timeout_ns;  // bound on every device-side wait
    int max_blocks;     // partials stride
    int resident;       // 1: an FP32 single-system run may keep each block's neighbourhood in shared memory
    int withhold;       // test hook: block 0 withholds its arrival at the launch's first grid barrier
    int tlog_every;     // > 0: the steps whose number is a multiple of it write a thermo-log record
    int uni;            // 1: uniform coefficients (see uni_swap / uni_other)
    int uni_swap;       // table index of the reactive pair coefficients (UNI)
    int uni_other;      // table index of the other pairs' coefficients (UNI)
    // Uniform coefficients ([0] reactive, [1] other), read by the kernels
    // straight from the kernel-parameter constant bank.
    PairP<float> uf[2];
    PairP<double> ud[2];
};

// Host-side launchers (defined once per precision).
template <typename Real>
cudaError_t launch_run(const Dev<Real>& d, const RunArgs& a, int grid, int block, cudaStream_t s);
template <typename Real>
cudaError_t run_occupancy(int block, int* blocks_per_sm);
// The 1024-thread step kernel (two-barrier step only), run by bonded networks.
template <typename Real>
cudaError_t launch_run_wide(const Dev<Real>& d, const RunArgs& a, int grid, cudaStream_t s);
template <typename Real>
cudaError_t run_occupancy_wide(int* blocks_per_sm);
// Batched launch (k_batch): per-system device structures and run arguments in
// device memory; block b runs items[item_ofs[b] .. item_ofs[b + 1]), each
// (system, rank in its group, group size, unused).  One launcher per block
// shape (threads per block): 1024 in both precisions, 512, 384 and 256 in FP32;
// batch_occupancy_<T> gives the blocks per SM of that shape.
template <typename Real>
struct Prec {};
#define SWP_DECLARE_BATCH(R, T)                                                                             \
    cudaError_t launch_batch_##T(const Dev<R>* devs, const RunArgs* args, const int* item_ofs,              \
                                 const int4* items, int uni, int bonds, int grid, cudaStream_t s);           \
    cudaError_t batch_occupancy_##T(Prec<R>, int* blocks_per_sm);
SWP_DECLARE_BATCH(float, 1024)
SWP_DECLARE_BATCH(double, 1024)
SWP_DECLARE_BATCH(float, 512)
SWP_DECLARE_BATCH(float, 384)
SWP_DECLARE_BATCH(float, 256)
// Derivatives with respect to one reactive type pair's (lambda, eps, sigma).
// theta: (lambda, eps, sigma) in device memory; pc < 0: the control block's
// current snapshot set; dU (device, may be null): dU/dtheta from the sums.
template <typename Real>
cudaError_t launch_param_grad(const Dev<Real>& d, int pc, double* sd, double* part, const double* theta,
                              double* out, double* total, double* dU, cudaStream_t s);
template <typename Real>
cudaError_t launch_eval_prep(const Dev<Real>& d, int ti, int tj, const double* theta, double c_rmin, double c_rb,
                             double rbond, const int* type, cudaStream_t s);
template <typename Real>
cudaError_t launch_set_state(const Dev<Real>& d, cudaStream_t s);
template <typename Real>
cudaError_t launch_get_state(const Dev<Real>& d, int pc, int ac, cudaStream_t s);
template <typename Real>
cudaError_t launch_get_forces(const Dev<Real>& d, int pc, cudaStream_t s);
template <typename Real>
cudaError_t launch_get_nlist(const Dev<Real>& d, int pc, int* rows, int* counts, int width,
                             cudaStream_t s);
template <typename Real>
size_t run_smem_bytes();

}  // namespace swp
