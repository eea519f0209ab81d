// Internal declarations shared by the host code and the kernels of the IREBM
// library.  Nothing here is part of the C ABI (see include/lbm_stefan.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Fixed-point accumulator for deterministic FP64 sums across thread blocks:
// the value is (hi * 2^64 + lo) * 2^-60 as a two's-complement 128-bit integer.
// Integer addition is associative, so the result does not depend on the
// order in which tiles add their partial sums.
struct Acc128 {
    unsigned long long lo;
    long long hi;
};

// Fixed-point accumulator of the per-step sums, updated with return-less
// atomic additions: the 128-bit two's-complement value is split into four
// 32-bit limbs, limb k being added into limb[k] (64 bits hold the sum of up to
// 2^32 limbs without overflow); the value is sum_k limb[k] * 2^(32k) modulo
// 2^128, formed with the carries when it is read.
struct AccSum {
    unsigned long long limb[4];
};

// One stripe of a step's sums.  The blocks of a launch add into
// kStripes stripes (block index mod kStripes), each on its own 128-byte line,
// so that their atomic additions are spread over the L2 slices; the stripes
// are summed when the step is published.
struct alignas(128) StepStripe {
    AccSum energy;                 // sum_x theta' + phi(theta')/Ste
    AccSum flux;                   // boundary flux
    unsigned long long newton;     // nodes that ran the Newton iteration
    unsigned long long iters;      // sum of their iteration counts
    unsigned long long liquid;     // saturated liquid nodes (each adds 1/Ste to the energy)
    unsigned long long dir[4];     // Dirichlet nodes per wall (each adds phi(theta_wall)/Ste)
    unsigned long long shifted;    // nodes whose energy term was added less the state's shift s
};
constexpr int kStripes = 32;

// Per-problem device statistics.  The "cur" stripes accumulate during one
// step launch; the last block of the launch publishes them and clears them.
struct DevStats {
    StepStripe cur[kStripes];
    int cur_maxit;                 // largest Newton iteration count
    int error;                     // sticky: lbm_status of a device-detected failure
    double energy, energy_prev, flux, imbalance, imbalance_max;
    long long steps;
    long long newton_nodes;
    long long newton_iters;        // sum of the Newton iteration counts of the last step
    int newton_max_iter;
    int have_energy;               // energy holds E(t) of the current state
    // adjoint accumulators: dL/dtheta_wall[4], dL/dSte, loss
    Acc128 g_wall[4];
    Acc128 g_ste;
    Acc128 loss;
};

// Device view of one problem.  Populations are stored as q planes (SoA);
// plane i starts at base + i * plane; each plane has ny + 2 rows of `pitch`
// elements, the first and last being zero halo rows, so row y (-1 .. ny)
// starts at (y + 1) * pitch.  pitch is a multiple of the warp segment width.
struct Problem {
    void* state[2];          // ping-pong population buffers
    long long tail_off;      // byte offset of each buffer's tail (after the planes); the tail of an
                             // FP32 D2Q9 / D2Q5 state holds the shift s (a float, the same in both
                             // buffers): the planes hold Omega_i - w_i s, so M0 = sum of the stored + s
    int nx, ny, pitch;
    int q;                   // 3 (D1Q3), 5 (D2Q5) or 9 (D2Q9)
    long long plane;         // elements per plane
    double omega;            // 1/tau
    double ste, inv_ste, delta, inv_delta;
    double tol;
    double sat;              // saturation threshold K*delta of the exact-source shortcut
    // constants of the mixed-precision Newton solve, converted on the host so
    // that a solve spends no FP64 instruction on them
    double inv_delta2, inv_delta3;
    float inv_ste_f, inv_delta_f, delta_f;
    float omega_f, omc_f, sat_f;   // (float) omega, (float)(1 - omega), (float) sat
    int maxit;
    int bb_mode;
    int wall_kind[4];        // W, E, S, N
    double wall_theta[4];
    double wall_tanh[4];     // tanh(theta_wall / delta), set on the device (wall_constants)
    double wall_phi[4];      // phi(theta_wall)
    float wall_th_hi[4];     // theta_wall as a float-float pair
    float wall_th_lo[4];
    float wall_slope[4];     // phi'(theta_wall)/Ste = (1 - tanh^2)/(2 delta Ste)
    float wall_dth_max;      // 1e-4 delta: range of the linear phi difference at a Dirichlet node
    int method;              // 0 IREBM (Algorithm 3), 1 EEBM (Algorithm 2), 2 ILFBM (Algorithm 1; FP64)
    double wall_H[4];        // EEBM: enthalpy of theta_wall, theta_wall + [theta_wall > 0]/Ste
    float wall_H_hi[4], wall_H_lo[4];
    int nseg, nstrip, tile_h;
    int tile0;               // first global tile index of this problem
    int ntiles;
    int stats;               // index into the DevStats array
};

// A node whose local Newton solve is deferred to the job kernel: the step
// kernel stores its q_i (not yet relaxed) and these inputs.
struct NewtonJob {
    int prob;                // problem index
    int node;                // y * nx + x
    double m0;               // M0(q) after the wall closures
    double theta;            // theta(t) = M0(f) at the node
    // FP32 form: m0 and theta are stored as float-float pairs (hi, lo) in the
    // bytes of m0 and theta, so the step kernel needs no FP64 conversion
};

// Per-launch arguments of the forward step kernels.
struct StepArgs {
    const Problem* probs;    // device array
    int nprob;
    const int2* schedule;    // device: (problem, local tile) per schedule slot; NULL = single problem
    int nslots;              // schedule length (total tiles)
    int parity;              // read state[parity], write state[parity ^ 1]
    double* rec;             // optional theta' record plane (single problem only), ny x pitch doubles
    DevStats* stats;
    unsigned int* ticket;    // last-block counter, zero between launches
    NewtonJob* jobs;         // deferred Newton nodes (D2Q9), capacity = total nodes
    unsigned int* job_count; // number of jobs; reset by the job kernel
    // FP32 D2Q9 flat step over several problems: one block per tile
    // (problem, 128-column strip, first of 8 rows) and one warp per wall row
    // (problem, 2 strip + (0: row 0, 1: row ny-1)); NULL: a single problem
    const int4* ftiles = nullptr;
    const int2* wrows = nullptr;
    int nwrows = 0;
    const int2* crows = nullptr;   // (problem, first row) per 32-row block of W / E groups
    // single problem: the flat kernel's strips seg0 .. seg0 + nsegc - 1 (nsegc 0: all)
    int seg0 = 0, nsegc = 0;
};

// TMA descriptors of the single-problem FP32 D2Q9 step: state[0], state[1]
// as 3-D tensors (column over `pitch`, row y + 1 over ny + 2 rows, plane
// 0..q-1); a load copies (kTmaW + 2 kTmaHalo) columns x 1 row x q planes.
constexpr int kTmaW = 128;               // columns per block (one node per consumer thread)
constexpr int kTmaHalo = 4;              // extra loaded columns on each side (16 bytes)
struct TmaMaps {
    CUtensorMap load[2];                 // single problem
    int nsegs;                           // pitch / kTmaW column strips (single problem)
    int nparts;                          // row ranges per strip; grid = nsegs * nparts
    long long wait_ns = 2000000000LL;    // bound of every wait on a row load, in nanoseconds
    int withhold_load = -1;              // test hook: >= 0 skips that row load of block 0 (0: the row
                                         // above its first row); -1: off
};

// Per-launch arguments of the Newton job kernel (runs after every D2Q9 step).
struct JobArgs {
    const Problem* probs;
    int nprob;
    int parity;              // the step read state[parity] and wrote state[parity ^ 1]
    double* rec;             // theta' record plane of the step (single problem), may be NULL
    DevStats* stats;
    unsigned int* ticket;
    const NewtonJob* jobs;
    unsigned int* job_count;
    int publish;             // 1: the last block publishes the step statistics; 0: it only clears the list
    // Two launches may share one list: with `cursor` set, each warp takes the
    // next 32 jobs of `jobs` from that counter (atomicAdd), so a launch that
    // starts late takes what an earlier one has not reached (every launch that
    // shares the cursor must start after the list is complete: a warp that
    // read a shorter count would claim jobs it then skips); without it the
    // warps take the list grid-stride.  `jobs2`: a second list, counted by
    // `job_count2`, that this launch alone solves (grid-stride) after the
    // first; a launch with `job_count2` set but no `jobs2` leaves it to the
    // other.  `nblocks`: the blocks of every launch that shares `ticket` (0:
    // this launch's grid); the last of them publishes and clears both counts
    // and the cursor (so each launch that shares the ticket carries both).
    unsigned int* cursor = nullptr;
    const NewtonJob* jobs2 = nullptr;
    unsigned int* job_count2 = nullptr;
    int nblocks = 0;
};

// Constants of the interior-node adjoint terms, converted once on the host.
struct AdjConst {
    float omc_f, om_f, inv_delta_f, inv_ste_f, inv_ste2_f, thr_f;
    double omc, om, inv_delta, inv_ste, thr;
};

// Per-launch arguments of the adjoint kernels (single problem).
struct AdjArgs {
    Problem pb;              // by value: read from the kernel parameter bank
    AdjConst c;
    const double* theta_t;   // recorded theta(t), ny x pitch
    const double* theta_t1;  // recorded theta(t+1), ny x pitch
    const void* adj_in;      // lambda(t+1), state layout
    void* adj_out;           // lambda(t), state layout
    DevStats* stats;
    int tile_h;              // rows per warp tile of the D2Q9 adjoint
    int ntiles;              // nseg * ceil(ny / tile_h)
    // plane i of adj_in / adj_out (D2Q9): kernel parameters, so that the
    // addresses come from the parameter bank instead of per-thread registers
    const void* in_plane[9];
    void* out_plane[9];
};

constexpr int kWarpsPerBlock = 4;
constexpr int kAdjTileH = 32;  // default rows per warp tile of the D2Q9 adjoint

// D2Q9 launchers (step_d2q9.cu)
cudaError_t launch_d2q9_step(int precision, const StepArgs& a, int grid, cudaStream_t s);
int d2q9_segment_width(int precision);   // nodes per warp segment
int d2q9_blocks_per_sm(int precision);   // resident step blocks per SM (persistent grid)
cudaError_t launch_d2q9_tma(const StepArgs& a, const TmaMaps& m, cudaStream_t s);
// single problem, FP32: the interior rows and the rows that touch a wall (two
// launches; with side, fork and join the second runs on `side`, joined back to s)
// FP32 D2Q9 flat step: the wall kernel (nwrows S / N rows, ncblocks blocks of
// W / E groups) and the flat kernel (nftiles blocks), both appending Newton
// nodes to a.jobs; the job kernel is the caller's.
cudaError_t launch_d2q9_flat(const StepArgs& a, int nftiles, int nwrows, int ncblocks, int method, cudaStream_t s);
int d2q9_tma_blocks_per_sm();
// q = 9 or 5; grid 0: two blocks per SM; prio != 0: that scheduling priority
// side: the launch beside the flat stencil kernel (kJobSideThreads per block), else 256
cudaError_t launch_newton_jobs(int precision, int q, const JobArgs& a, cudaStream_t s, int grid = 0, int prio = 0,
                               bool side = false);

// D2Q5 launchers (step_d2q5.cu): one tile per warp over a.nslots tiles
cudaError_t launch_d2q5_step(int precision, const StepArgs& a, cudaStream_t s);
int d2q5_segment_width(int precision);   // nodes per warp segment

// D1Q3 launchers (step_d1q3.cu)
cudaError_t launch_d1q3_step(int precision, const StepArgs& a, const Problem& hp, cudaStream_t s);
cudaError_t launch_d1q3_fused(int precision, const StepArgs& a, const Problem& hp, int nsteps, int start_parity,
                              double* rec, cudaStream_t s);
bool d1q3_fused_fits(int precision, int nx);

// ILFBM (Algorithm 1) on D1Q3, FP64, one block over the whole lattice (ilfbm.cu)
cudaError_t launch_ilfbm_d1q3(const StepArgs& a, const Problem& hp, int nsteps, cudaStream_t s);
bool ilfbm_d1q3_fits(int nx);
// one ILFBM step on D2Q9 / D2Q5 (hp.q), FP64: scratch holds 5 nx*ny doubles,
// flags 5 unsigned ints; publishes the step statistics (hp: the host copy, passed by value)
cudaError_t launch_ilfbm_2d(const Problem& hp, int parity, double* scratch,
                            unsigned int* flags, DevStats* stats, unsigned int* ticket, cudaStream_t s);

// Field and state kernels (fields.cu)
cudaError_t launch_init_state(int precision, const Problem* dprob, const Problem& hp, const double* theta0,
                              int parity, DevStats* st, cudaStream_t s);
cudaError_t launch_front(int precision, const Problem* dprob, const Problem& hp, int parity, int wall, double* out,
                         cudaStream_t s);
cudaError_t launch_fields(int precision, const Problem* dprob, const Problem& hp, int parity, double* theta,
                          double* phi, double* H, double* theta_plane, cudaStream_t s);
cudaError_t launch_finalize_init(DevStats* st, cudaStream_t s);
// tanh(theta_wall/delta) and phi(theta_wall) of every wall, for nprob problems
cudaError_t launch_wall_constants(Problem* dprobs, int nprob, cudaStream_t s);

// Adjoint kernels (adjoint.cu)
cudaError_t launch_adj_seed(int precision, const Problem* dprob, const Problem& hp, const double* theta_T,
                            const double* phi_target, void* adj, DevStats* st, cudaStream_t s);
cudaError_t launch_adj_step(int precision, const AdjArgs& a, const Problem& hp, cudaStream_t s);
cudaError_t launch_adj_finish(int precision, const Problem* dprob, const Problem& hp, const void* adj0,
                              double* g_theta0, DevStats* st, cudaStream_t s);

}  // namespace lbm
