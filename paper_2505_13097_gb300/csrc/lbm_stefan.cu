// Host side of the C ABI declared in include/lbm_stefan.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lbm_stefan.h"
#include "lbm_internal.h"

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#ifndef LBM_PLANE_PAD
#define LBM_PLANE_PAD 0
#endif

using lbm::DevStats;
using lbm::Problem;
using lbm::StepArgs;

namespace {

thread_local char g_err[512] = "";

lbm_status fail(lbm_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

#define CUDA_TRY(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// NVTX range for the lifetime of the object (visible to Nsight tools when one
// is attached; the header-only NVTX API does nothing otherwise)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Steps per captured CUDA graph (an even number, so a graph starts and ends on parity 0).
constexpr int kGraphSteps = 32;

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int steps = 0;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        steps = 0;
    }
};

}  // namespace

struct lbm_stefan {
    lbm_stefan_params p;
    Problem hp;
    Problem* dprob = nullptr;
    int precision = 0;
    size_t elem = 8;
    size_t state_bytes = 0;
    cudaStream_t stream = nullptr;
    DevStats* dstats = nullptr;
    unsigned int* dticket = nullptr;
    double* dscratch = nullptr;   // 3 * nx * ny doubles (host field transfers)
    lbm::NewtonJob* djobs = nullptr;    // deferred Newton nodes of one step (capacity nx * ny)
    unsigned int* djob_count = nullptr;
    int parity = 0;
    bool ic = false;
    int adj_tile_h = lbm::kAdjTileH;   // rows per warp tile of the D2Q9 adjoint
    unsigned int* dilf = nullptr;      // 2D ILFBM: inner-loop flags (done, iteration, changed x 3)
    double* dilf_scratch = nullptr;    // 2D ILFBM: S0, two l iterates, two l differences (5 nx*ny)
    bool flat = false;                 // FP32 D2Q9: the flat and wall kernels
    bool use_tma = false;              // FP32 D2Q9: the TMA row-pipeline kernel (for the wait test hook)
    lbm::TmaMaps tma;
    int withhold_load = -1;            // test hook of the TMA kernel's row loads (-1: off)
    cudaStream_t side = nullptr;       // split FP32 D2Q9 step: stream of the left half's Newton solves
    cudaEvent_t ev_fork = nullptr, ev_half = nullptr, ev_join = nullptr;
    cudaEvent_t ev_walls = nullptr;   // split step: the wall kernels are done (list A's wall part is final)
    GraphCache graph;
    // captured adjoint segments (lbm_stefan_adjoint_segment): recompute + reverse
    // steps for one (length, trajectory, adjoint buffers) combination each
    struct SegGraph {
        int n;
        const void* traj;
        const void* a;
        const void* b;
        cudaGraphExec_t exec;
    };
    std::vector<SegGraph> seg_graphs;
    void reset_seg_graphs()
    {
        for (auto& g : seg_graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        seg_graphs.clear();
    }
};

struct lbm_stefan_batch {
    int count = 0;
    int precision = 1;
    size_t elem = 4;
    std::vector<Problem> hp;
    std::vector<size_t> state_bytes;
    Problem* dprobs = nullptr;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    DevStats* dstats = nullptr;
    unsigned int* dticket = nullptr;
    int2* dsched = nullptr;
    int nslots = 0;
    int tile_h = 16;
    int schedule = 1;
    int grid = 0;
    int parity = 0;
    cudaStream_t stream = nullptr;
    double* dscratch = nullptr;
    size_t scratch_elems = 0;
    lbm::NewtonJob* djobs = nullptr;
    unsigned int* djob_count = nullptr;
    bool use_flat = false;             // FP32: the flat and wall-row kernels over tables
    int4* dftiles = nullptr;           // (problem, strip, first row) per flat block
    int nftiles = 0;
    int2* dwrows = nullptr;            // (problem, 2 strip + S/N) per wall row
    int nwrows = 0;
    int2* dcrows = nullptr;            // (problem, first row) per 32-row block of W / E groups
    int ncblocks = 0;
    int nftiles_left = 0;              // the tiles of the problems' left halves come first
    size_t total_nodes = 0;
    cudaStream_t side = nullptr;       // split step (stream of its own): the left halves' Newton solves
    cudaEvent_t ev_fork = nullptr, ev_half = nullptr, ev_join = nullptr;
    cudaEvent_t ev_walls = nullptr;   // split step: the wall kernels are done (list A's wall part is final)
    GraphCache graph;
};

// ------------------------------------------------------------------ helpers

static lbm_status validate_common(int nx, int ny, double tau, double delta, double ste, double tol, int maxit)
{
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2 (got %g)", tau);
    if (!(delta > 0.0) || !std::isfinite(delta)) return fail(LBM_ERR_ARG, "delta must be > 0 (got %g)", delta);
    if (!(ste > 0.0) || !std::isfinite(ste)) return fail(LBM_ERR_ARG, "Ste must be > 0 (got %g)", ste);
    if (!(tol > 0.0) || maxit < 1) return fail(LBM_ERR_ARG, "newton_tol must be > 0 and newton_max_iter >= 1");
    if (nx < 2 || ny < 1) return fail(LBM_ERR_ARG, "nx must be >= 2 (got %d, %d)", nx, ny);
    return LBM_OK;
}

// Threshold of the exact-source shortcut: theta and m0 beyond K*delta on the same
// side give theta' = m0.  FP64: K = 19.5, where tanh rounds to +-1 and the
// shortcut is exact.  FP32 populations: K with 2 exp(-2K)/Ste = 1e-10 (the
// neglected source), about 100x below the rounding of the stored populations.
static double saturation_threshold(int precision, double delta, double ste)
{
    double k = 19.5;
    if (precision == LBM_FP32) k = std::min(19.5, std::max(10.0, 0.5 * std::log(2.0 / (ste * 1e-10))));
    return k * delta;
}

// Rows per warp tile of the D2Q9 adjoint: the tallest of 32, 16, 8, 4 that
// still gives four warp tiles per resident warp slot (16 per SM).  Each tile
// also evaluates the row below and above it, so tall tiles waste less.
#ifndef LBM_ADJ_TILE_H
#define LBM_ADJ_TILE_H 0
#endif
static int adjoint_tile_h(const Problem& hp)
{
    if (LBM_ADJ_TILE_H > 0) return LBM_ADJ_TILE_H;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 152;
    const long long want = 4LL * 16 * sms;
    int th = lbm::kAdjTileH;
    while (th > 4 && (long long)hp.nseg * ((hp.ny + th - 1) / th) < want) th /= 2;
    return th;
}

static void fill_problem(Problem& pb, int q, int nx, int ny, int pitch, double tau, double delta, double ste,
                         double tol, int maxit, int bb_mode, int tile_h, int segw, int precision)
{
    std::memset(&pb, 0, sizeof pb);
    pb.nx = nx;
    pb.ny = ny;
    pb.q = q;
    pb.pitch = pitch;
    // planes one stride apart (+ LBM_PLANE_PAD elements) so that the nine
    // streams of a step do not fall on the same memory partitions
    pb.plane = (long long)(ny + 2) * pitch + LBM_PLANE_PAD;
    pb.omega = 1.0 / tau;
    pb.ste = ste;
    pb.inv_ste = 1.0 / ste;
    pb.delta = delta;
    pb.inv_delta = 1.0 / delta;
    pb.tol = tol;
    pb.inv_delta2 = pb.inv_delta * pb.inv_delta;
    pb.inv_delta3 = pb.inv_delta2 * pb.inv_delta;
    pb.inv_ste_f = (float)pb.inv_ste;
    pb.inv_delta_f = (float)pb.inv_delta;
    pb.delta_f = (float)delta;
    pb.sat = saturation_threshold(precision, delta, ste);
    pb.omega_f = (float)pb.omega;
    pb.omc_f = (float)(1.0 - pb.omega);
    pb.sat_f = (float)pb.sat;
    pb.maxit = maxit;
    pb.bb_mode = bb_mode;
    pb.tile_h = tile_h;
    pb.nseg = pitch / segw;
    pb.nstrip = (ny + tile_h - 1) / tile_h;
    pb.ntiles = pb.nseg * pb.nstrip;
    // the planes (D1Q3: a fourth, the ILFBM liquid fraction), then the tail
    pb.tail_off = (long long)(q == 3 ? 4 : q) * pb.plane * (precision == LBM_FP32 ? 4 : 8);
}

// Bytes after the planes of a state buffer: the shift of an FP32 D2Q9 / D2Q5
// state (a float; zero otherwise), in a block of its own.
constexpr size_t kStateTail = 256;

static lbm_status upload_problem(lbm_stefan* h)
{
    CUDA_TRY(cudaMemcpyAsync(h->dprob, &h->hp, sizeof(Problem), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(lbm::launch_wall_constants(h->dprob, 1, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

static StepArgs single_args(lbm_stefan* h, int parity, double* rec)
{
    StepArgs a;
    a.probs = h->dprob;
    a.nprob = 1;
    a.schedule = nullptr;
    a.nslots = h->hp.ntiles;
    a.parity = parity;
    a.rec = rec;
    a.stats = h->dstats;
    a.ticket = h->dticket;
    a.jobs = h->djobs;
    a.job_count = h->djob_count;
    return a;
}

static lbm::JobArgs job_args(const Problem* probs, int nprob, int parity, double* rec, DevStats* st,
                             unsigned int* ticket, lbm::NewtonJob* jobs, unsigned int* count)
{
    lbm::JobArgs j;
    j.probs = probs;
    j.nprob = nprob;
    j.parity = parity;
    j.rec = rec;
    j.stats = st;
    j.ticket = ticket;
    j.jobs = jobs;
    j.job_count = count;
    j.publish = 1;
    return j;
}

#ifndef LBM_SPLIT
#define LBM_SPLIT 1   // FP32 D2Q9 on a stream of its own: the left strips' Newton solves beside the right strips
#endif

// The two job lists of a split FP32 D2Q9 step: list A (the wall kernel's and
// the left strips' nodes) from djobs, list B (the right strips') after it.
static size_t split_cap_a(const Problem& hp)
{
    const int nsegs = hp.pitch / lbm::kTmaW;
    return (size_t)(nsegs / 2) * lbm::kTmaW * hp.ny + 2 * (size_t)hp.pitch + 8 * (size_t)hp.ny;
}

static cudaError_t launch_flat_final_jobs(lbm_stefan* h, const StepArgs& a);

// FP32 D2Q9 single-problem step: the nodes on or next to a wall (the wall
// kernels), rows 1 .. ny-2 of every 128-column strip (the flat kernel), then
// the Newton job kernel.  With a side stream the strips are cut into a left
// and a right half.  List A holds the Newton nodes of the wall kernels and of
// the left half, list B those of the right half.  On the side stream, job
// blocks (one per SM, at a higher priority) take list A from a shared cursor
// while the right half streams.  After the right half, a full job launch takes what is left of
// list A, then list B (it waits for the wall kernels, whose nodes are part of
// list A); the last block of the two launches publishes the step.
// The side stream joins the main one at the end.  Which launch solves a node
// does not change its result.
// final_jobs = false leaves out the last job launch (step_timed times it) and
// joins before it; fev (step_timed): four events recorded on the handle's
// stream before and after the flat launches (left half, right half; one
// launch without a split).
static lbm::JobArgs split_jobs_first(const Problem* probs, int nprob, int parity, double* rec, DevStats* st,
                                     unsigned int* ticket, lbm::NewtonJob* jobs, unsigned int* counts, int nblocks)
{
    lbm::JobArgs j = job_args(probs, nprob, parity, rec, st, ticket, jobs, counts);
    j.cursor = counts + 2;
    j.job_count2 = counts + 1;   // cleared by whichever launch ends last
    j.nblocks = nblocks;
    return j;
}

static lbm::JobArgs split_jobs_last(const lbm::JobArgs& first, lbm::NewtonJob* jobs_b)
{
    lbm::JobArgs j = first;
    j.jobs2 = jobs_b;
    return j;
}

// Blocks of the single problem's side Newton launch: one per SM.  Each takes
// the place of one of the flat kernel's three blocks on its SM while it runs;
// the FP64 refinement of the solves keeps the band's work on the FP64 pipe, so
// fewer side blocks would leave more of list A to the last job launch, after
// the streaming.
static int split_side_blocks(int sms) { return sms > 0 ? sms : 1; }

static int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

static cudaError_t launch_flat(lbm_stefan* h, const StepArgs& a, bool final_jobs = true, cudaEvent_t* fev = nullptr)
{
    const int nsegs = h->hp.pitch / lbm::kTmaW;
    const int nbands = h->hp.ny > 2 ? (h->hp.ny + 7) / 8 : 0;
    const int ncblocks = h->hp.ny > 2 ? (h->hp.ny - 2 + 31) / 32 : 0;
    const int half = nsegs / 2;
    cudaError_t e;
    if (!(h->side && half >= 1 && nbands > 0)) {
        // the wall kernels, then the flat kernel
        e = lbm::launch_d2q9_flat(a, 0, 2 * nsegs, ncblocks, h->hp.method, h->stream);
        if (e == cudaSuccess && fev) e = cudaEventRecord(fev[0], h->stream);
        if (e == cudaSuccess) e = lbm::launch_d2q9_flat(a, nsegs * nbands, 0, 0, h->hp.method, h->stream);
        if (e == cudaSuccess && fev) e = cudaEventRecord(fev[1], h->stream);
        if (e == cudaSuccess && fev) e = cudaEventRecord(fev[2], h->stream);
        if (e == cudaSuccess && fev) e = cudaEventRecord(fev[3], h->stream);
        if (e != cudaSuccess || !final_jobs) return e;
        return lbm::launch_newton_jobs(1, 9, job_args(h->dprob, 1, a.parity, a.rec, h->dstats, h->dticket, h->djobs,
                                                      h->djob_count),
                                       h->stream);
    }
    int least = 0, prio = 0;
    const int sms = device_sms();
    e = sms > 0 ? cudaDeviceGetStreamPriorityRange(&least, &prio) : cudaErrorInvalidDevice;
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    if (e == cudaSuccess) e = lbm::launch_d2q9_flat(a, 0, 2 * nsegs, ncblocks, h->hp.method, h->side);   // list A
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_walls, h->side);
    StepArgs aa = a;   // list A: djobs, counter 0
    aa.seg0 = 0;
    aa.nsegc = half;
    if (e == cudaSuccess && fev) e = cudaEventRecord(fev[0], h->stream);
    if (e == cudaSuccess) e = lbm::launch_d2q9_flat(aa, half * nbands, 0, 0, h->hp.method, h->stream);
    if (e == cudaSuccess && fev) e = cudaEventRecord(fev[1], h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_half, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_half, 0);
    if (e != cudaSuccess) return e;
    const lbm::JobArgs ja =
        split_jobs_first(h->dprob, 1, a.parity, a.rec, h->dstats, h->dticket, h->djobs, h->djob_count,
                         split_side_blocks(sms) + sms);
    e = lbm::launch_newton_jobs(1, 9, ja, h->side, split_side_blocks(sms), prio, true);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
    if (e != cudaSuccess) return e;
    StepArgs ab = a;   // list B: after list A, counter 1
    ab.jobs = h->djobs + split_cap_a(h->hp);
    ab.job_count = h->djob_count + 1;
    ab.seg0 = half;
    ab.nsegc = nsegs - half;
    if (fev) e = cudaEventRecord(fev[2], h->stream);
    if (e == cudaSuccess) e = lbm::launch_d2q9_flat(ab, (nsegs - half) * nbands, 0, 0, h->hp.method, h->stream);
    if (e == cudaSuccess && fev) e = cudaEventRecord(fev[3], h->stream);
    if (e != cudaSuccess) return e;
    if (!final_jobs) return cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    // the last job launch reads list A's count and takes the rest of it: the
    // wall kernels (side stream) must have appended their nodes
    e = cudaStreamWaitEvent(h->stream, h->ev_walls, 0);
    if (e == cudaSuccess) e = launch_flat_final_jobs(h, a);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    return e;
}

// The last job launch of a flat step (after launch_flat(h, a, false)).
static cudaError_t launch_flat_final_jobs(lbm_stefan* h, const StepArgs& a)
{
    const int nsegs = h->hp.pitch / lbm::kTmaW;
    const bool split = h->side && nsegs / 2 >= 1 && h->hp.ny > 2;
    const int sms = device_sms();
    if (sms <= 0) return cudaErrorInvalidDevice;
    if (!split)
        return lbm::launch_newton_jobs(1, 9, job_args(h->dprob, 1, a.parity, a.rec, h->dstats, h->dticket, h->djobs,
                                                      h->djob_count),
                                       h->stream);
    const lbm::JobArgs ja =
        split_jobs_first(h->dprob, 1, a.parity, a.rec, h->dstats, h->dticket, h->djobs, h->djob_count,
                         split_side_blocks(sms) + sms);
    return lbm::launch_newton_jobs(1, 9, split_jobs_last(ja, h->djobs + split_cap_a(h->hp)), h->stream,
                                   sms);
}

// One step.  D2Q9 and D2Q5: the stream/collide kernel(s), which defer the
// nodes that need the Newton iteration, then the job kernel that solves them
// (FP32 D2Q9: the wall-row kernel and the flat kernel, three launches in all;
// FP64 D2Q9 and D2Q5: two).  D1Q3: one launch.  While the wait test hook is
// on, the FP32 D2Q9 step runs the TMA row-pipeline kernel instead of the
// flat pair (the kernel with the waits the hook exercises).
static cudaError_t launch_one(lbm_stefan* h, int parity, double* rec)
{
    StepArgs a = single_args(h, parity, rec);
    if (h->p.lattice == LBM_D2Q5) {
        const cudaError_t e = lbm::launch_d2q5_step(h->precision, a, h->stream);
        if (e != cudaSuccess) return e;
        return lbm::launch_newton_jobs(h->precision, 5,
                                       job_args(h->dprob, 1, parity, rec, h->dstats, h->dticket, h->djobs, h->djob_count),
                                       h->stream);
    }
    if (h->p.lattice == LBM_D2Q9) {
        cudaError_t e;
        if (h->flat && h->withhold_load < 0) return launch_flat(h, a);   // with its job kernels
        if (h->use_tma) {
            e = lbm::launch_d2q9_tma(a, h->tma, h->stream);
        } else {
            // one tile per warp; the hardware scheduler balances the short tiles
            const int grid = (h->hp.ntiles + lbm::kWarpsPerBlock - 1) / lbm::kWarpsPerBlock;
            e = lbm::launch_d2q9_step(h->precision, a, grid, h->stream);
        }
        if (e != cudaSuccess) return e;
        return lbm::launch_newton_jobs(h->precision, h->hp.q,
                                       job_args(h->dprob, 1, parity, rec, h->dstats, h->dticket, h->djobs, h->djob_count),
                                       h->stream);
    }
    return lbm::launch_d1q3_step(h->precision, a, h->hp, h->stream);
}

static lbm_status check_stats_error(lbm_stefan* h, DevStats* out)
{
    DevStats st;
    CUDA_TRY(cudaMemcpyAsync(&st, h->dstats, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (out) *out = st;
    if (st.error) return fail((lbm_status)st.error, "device reported error %d (Newton limit or non-finite value)", st.error);
    return LBM_OK;
}

static double acc_host(const lbm::Acc128& a) { return (double)a.hi * 16.0 + (double)a.lo * 0x1p-60; }

// ------------------------------------------------------------------ one problem

// ------------------------------------------------------------------ TMA descriptors
#ifndef LBM_USE_TMA
#define LBM_USE_TMA 1
#endif
#ifndef LBM_TMA_ROWS
#define LBM_TMA_ROWS 16   // rows per block of the TMA step kernel
#endif

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// The q planes of one FP32 state buffer as a tensor (column, row incl. the
// two ghost rows, plane); box_x columns x 1 row x q planes per copy.
static bool encode_state_map(CUtensorMap* m, void* base, const Problem& hp, int box_x)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)hp.pitch, (cuuint64_t)hp.ny + 2, (cuuint64_t)hp.q};
    const cuuint64_t strides[2] = {(cuuint64_t)hp.pitch * 4, (cuuint64_t)hp.plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, 1, (cuuint32_t)hp.q};
    const cuuint32_t elem[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row stride of a single problem's state: whole kernel segments; FP32 D2Q9
// rows hold whole 128-column strips of the TMA step kernel.
static int state_pitch(int lattice, int precision, int nx)
{
    if (lattice == LBM_D1Q3) return round_up(nx, 32);
    if (lattice == LBM_D2Q5) return round_up(nx, lbm::d2q5_segment_width(precision));
    const int segw = lbm::d2q9_segment_width(precision);
    return round_up(nx, precision == LBM_FP32 ? std::max(segw, lbm::kTmaW) : segw);
}

// Descriptors and grid of the TMA step kernel; false leaves the warp-tile kernel in use.
static bool setup_tma(lbm_stefan* h)
{
    const Problem& hp = h->hp;
    if (hp.pitch % lbm::kTmaW != 0 || (hp.plane * 4) % 16 != 0) return false;
    for (int k = 0; k < 2; ++k)
        if (!encode_state_map(&h->tma.load[k], hp.state[k], hp, lbm::kTmaW + 2 * lbm::kTmaHalo)) return false;
    h->tma.nsegs = hp.pitch / lbm::kTmaW;
    // short row ranges: many blocks in flight hide the latency of each block's
    // row chain (measured: 16 rows beat 8, 32, 64 and one range per SM slot)
    h->tma.nparts = std::max(1, (hp.ny + LBM_TMA_ROWS - 1) / LBM_TMA_ROWS);
    const int per_sm = lbm::d2q9_tma_blocks_per_sm();   // also selects the shared-memory carveout
#ifdef LBM_TMA_VERBOSE
    fprintf(stderr, "tma: blocks/SM %d nsegs %d nparts %d\n", per_sm, h->tma.nsegs, h->tma.nparts);
#endif
    return per_sm > 0;
}

extern "C" lbm_status lbm_stefan_create(const lbm_stefan_params* p, void* cuda_stream, lbm_stefan** out)
{
    if (!p || !out) return fail(LBM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (p->lattice != LBM_D1Q3 && p->lattice != LBM_D2Q9 && p->lattice != LBM_D2Q5)
        return fail(LBM_ERR_ARG, "lattice must be D1Q3, D2Q9 or D2Q5");
    if (p->precision != LBM_FP64 && p->precision != LBM_FP32) return fail(LBM_ERR_ARG, "precision must be FP64 or FP32");
    if (p->bb_mode != LBM_BB_MIRROR && p->bb_mode != LBM_BB_LINK && p->bb_mode != LBM_NEU_EQ17)
        return fail(LBM_ERR_ARG, "bb_mode must be 0, 1 or 2");
    if (p->bb_mode == LBM_NEU_EQ17 && p->lattice != LBM_D2Q5)
        return fail(LBM_ERR_ARG, "the Neumann closure of Eq. (17) is the D2Q5 one");
    lbm_status s = validate_common(p->nx, p->ny, p->tau, p->delta, p->ste, p->newton_tol, p->newton_max_iter);
    if (s != LBM_OK) return s;
    if (p->lattice == LBM_D1Q3 && p->ny != 1) return fail(LBM_ERR_ARG, "D1Q3 needs ny = 1");
    if (p->lattice == LBM_D2Q9 && p->ny < 2) return fail(LBM_ERR_ARG, "D2Q9 needs ny >= 2");
    if (p->lattice == LBM_D2Q5 && (p->nx < 3 || p->ny < 3)) return fail(LBM_ERR_ARG, "D2Q5 needs nx, ny >= 3");
    if ((long long)p->nx * p->ny > (1ll << 31)) return fail(LBM_ERR_ARG, "more than 2^31 nodes");

    lbm_stefan* h = new lbm_stefan();
    h->p = *p;
    h->precision = p->precision;
    h->elem = p->precision == LBM_FP32 ? 4 : 8;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    const int q = p->lattice == LBM_D2Q9 ? 9 : (p->lattice == LBM_D2Q5 ? 5 : 3);
    const int segw = p->lattice == LBM_D2Q9   ? lbm::d2q9_segment_width(p->precision)
                     : p->lattice == LBM_D2Q5 ? lbm::d2q5_segment_width(p->precision)
                                              : 32;
    const bool tma = LBM_USE_TMA && p->lattice == LBM_D2Q9 && p->precision == LBM_FP32;
    const int pitch = state_pitch(p->lattice, p->precision, p->nx);
    fill_problem(h->hp, q, p->nx, p->ny, pitch, p->tau, p->delta, p->ste, p->newton_tol, p->newton_max_iter,
                 p->bb_mode, 16, segw, p->precision);
    // D1Q3: a fourth plane holds the liquid fraction of ILFBM (Algorithm 1), zero otherwise
    h->state_bytes = (size_t)h->hp.tail_off + kStateTail;
    cudaError_t e = cudaSuccess;
    void* bufs[2] = {nullptr, nullptr};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&bufs[k], h->state_bytes);
        if (e == cudaSuccess) e = cudaMemset(bufs[k], 0, h->state_bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->dprob, sizeof(Problem));
    if (e == cudaSuccess) e = cudaMalloc(&h->dstats, sizeof(DevStats));
    if (e == cudaSuccess) e = cudaMemset(h->dstats, 0, sizeof(DevStats));
    // [0]: the step's job list and job kernel; [1]: the split step's second list
    if (e == cudaSuccess) e = cudaMalloc(&h->dticket, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(h->dticket, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&h->dscratch, sizeof(double) * 3 * (size_t)p->nx * p->ny);
    if (e == cudaSuccess) e = cudaMalloc(&h->djob_count, 3 * sizeof(unsigned int));   // lists A, B; cursor of A
    if (e == cudaSuccess && q == 9) h->adj_tile_h = adjoint_tile_h(h->hp);
    if (e == cudaSuccess) e = cudaMemset(h->djob_count, 0, 3 * sizeof(unsigned int));
    h->hp.state[0] = bufs[0];
    h->hp.state[1] = bufs[1];
    h->hp.stats = 0;
    h->flat = p->lattice == LBM_D2Q9 && p->precision == LBM_FP32;
    if (e == cudaSuccess && tma) h->use_tma = setup_tma(h);
    // the split FP32 step (non-default streams only: the legacy stream would
    // serialize with its side stream), side stream of the highest priority
    if (e == cudaSuccess && h->flat && LBM_SPLIT && h->stream != nullptr) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_half, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_walls, cudaEventDisableTiming);
    }
    // the list of deferred Newton nodes (D2Q9, D2Q5): one job per node at most
    // (split FP32 step: two lists, the first with room for the wall kernel's
    // and the left half's nodes)
    const size_t njobs = h->side ? split_cap_a(h->hp) + (size_t)(h->hp.pitch / lbm::kTmaW - h->hp.pitch / lbm::kTmaW / 2) *
                                                            lbm::kTmaW * p->ny
                                 : (size_t)p->nx * p->ny;
    if (e == cudaSuccess && q != 3) e = cudaMalloc(&h->djobs, sizeof(lbm::NewtonJob) * njobs);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        lbm_stefan_destroy(h);
        return fail(LBM_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(e));
    }
    s = upload_problem(h);
    if (s != LBM_OK) {
        lbm_stefan_destroy(h);
        return s;
    }
    *out = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_set_bc(lbm_stefan* h, int wall, int kind, double theta_wall)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (wall < 0 || wall > 3) return fail(LBM_ERR_ARG, "wall must be 0..3");
    if (h->p.lattice == LBM_D1Q3 && wall > 1) return fail(LBM_ERR_ARG, "D1Q3 has only the W and E walls");
    if (kind != LBM_ADIABATIC && kind != LBM_DIRICHLET) return fail(LBM_ERR_ARG, "kind must be 0 or 1");
    if (!std::isfinite(theta_wall)) return fail(LBM_ERR_ARG, "theta_wall must be finite");
    h->hp.wall_kind[wall] = kind;
    h->hp.wall_theta[wall] = theta_wall;
    h->graph.reset();
    h->reset_seg_graphs();
    return upload_problem(h);
}

extern "C" lbm_status lbm_stefan_set_ste(lbm_stefan* h, double ste)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (!(ste > 0.0) || !std::isfinite(ste)) return fail(LBM_ERR_ARG, "Ste must be > 0 (got %g)", ste);
    h->p.ste = ste;
    h->hp.ste = ste;
    h->hp.inv_ste = 1.0 / ste;
    h->hp.inv_ste_f = (float)h->hp.inv_ste;
    h->hp.sat = saturation_threshold(h->precision, h->hp.delta, ste);
    h->hp.sat_f = (float)h->hp.sat;
    h->graph.reset();
    h->reset_seg_graphs();
    return upload_problem(h);
}

extern "C" lbm_status lbm_stefan_set_method(lbm_stefan* h, int method)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (method != LBM_IREBM && method != LBM_EEBM && method != LBM_ILFBM)
        return fail(LBM_ERR_ARG, "method must be 0 (IREBM), 1 (EEBM) or 2 (ILFBM)");
    // EEBM: D1Q3, D2Q9 and D2Q5 (every closure); the no-allocation step and batches stay IREBM
    if (method == LBM_ILFBM) {
        if (h->precision != LBM_FP64) return fail(LBM_ERR_ARG, "ILFBM is implemented in FP64");
        if (h->p.bb_mode == LBM_NEU_EQ17) return fail(LBM_ERR_ARG, "ILFBM uses the bounce-back closures");
        if (h->p.lattice == LBM_D1Q3 && !lbm::ilfbm_d1q3_fits(h->hp.nx))
            return fail(LBM_ERR_ARG, "ILFBM on D1Q3 holds the lattice in one block: at most 2,844 nodes");
        if (h->p.lattice != LBM_D1Q3) {
            // the liquid fraction needs a plane of its own after the q populations
            const size_t need = (size_t)(h->hp.q + 1) * h->hp.plane * h->elem + kStateTail;
            if (h->state_bytes < need) {
                void* nb[2] = {nullptr, nullptr};
                cudaError_t e = cudaSuccess;
                for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                    e = cudaMalloc(&nb[k], need);
                    if (e == cudaSuccess) e = cudaMemset(nb[k], 0, need);
                }
                if (e != cudaSuccess) {
                    cudaFree(nb[0]);
                    cudaFree(nb[1]);
                    return fail(LBM_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(e));
                }
                CUDA_TRY(cudaStreamSynchronize(h->stream));   // no step still reads the old buffers
                cudaFree(h->hp.state[0]);
                cudaFree(h->hp.state[1]);
                h->hp.state[0] = nb[0];
                h->hp.state[1] = nb[1];
                h->state_bytes = need;
                h->hp.tail_off = (long long)(need - kStateTail);
            }
            if (!h->dilf) CUDA_TRY(cudaMalloc(&h->dilf, 8 * sizeof(unsigned int)));
            if (!h->dilf_scratch)
                CUDA_TRY(cudaMalloc(&h->dilf_scratch, 5 * sizeof(double) * (size_t)h->hp.nx * h->hp.ny));
        }
    }
    h->hp.method = method;
    h->ic = false;   // the state of one method is not a state of the other
    h->graph.reset();
    h->reset_seg_graphs();
    return upload_problem(h);
}

extern "C" lbm_status lbm_stefan_set_ic(lbm_stefan* h, const double* theta0, int on_device)
{
    if (!h || !theta0) return fail(LBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->hp.nx * h->hp.ny;
    const double* src = theta0;
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(h->dscratch, theta0, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        src = h->dscratch;
    }
    CUDA_TRY(cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream));
    CUDA_TRY(lbm::launch_init_state(h->precision, h->dprob, h->hp, src, 0, h->dstats, h->stream));
    CUDA_TRY(lbm::launch_finalize_init(h->dstats, h->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->parity = 0;
    h->ic = true;
    return LBM_OK;
}

static lbm_status capture_graph(lbm_stefan* h)
{
    h->graph.reset();
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = launch_one(h, k & 1, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(LBM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    // per-node priorities: the split step's side Newton launch keeps its higher priority
    e = cudaGraphInstantiate(&h->graph.exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    h->graph.steps = kGraphSteps;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_step(lbm_stefan* h, int nsteps)
{
    NvtxRange r("lbm_stefan_step");
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (!h->ic) return fail(LBM_ERR_STATE, "set_ic must come before step");
    if (nsteps == 0) return LBM_OK;
    if (h->hp.method == LBM_ILFBM && h->p.lattice == LBM_D1Q3) {
        // all steps in one launch (one block over the lattice, whose barriers
        // separate the inner iterations)
        StepArgs a = single_args(h, h->parity, nullptr);
        CUDA_TRY(lbm::launch_ilfbm_d1q3(a, h->hp, nsteps, h->stream));
        h->parity ^= nsteps & 1;
        return LBM_OK;
    }
    if (h->hp.method == LBM_ILFBM) {
        // 2D: one launch per inner iteration (newton_max_iter of them, those
        // after convergence return at once), framed by the collision and the
        // final streaming
        for (int k = 0; k < nsteps; ++k) {
            CUDA_TRY(lbm::launch_ilfbm_2d(h->hp, h->parity, h->dilf_scratch, h->dilf, h->dstats, h->dticket,
                                          h->stream));
            h->parity ^= 1;
        }
        return LBM_OK;
    }
    if (h->p.lattice == LBM_D1Q3 && lbm::d1q3_fused_fits(h->precision, h->hp.nx)) {
        StepArgs a = single_args(h, h->parity, nullptr);
        CUDA_TRY(lbm::launch_d1q3_fused(h->precision, a, h->hp, nsteps, h->parity, nullptr, h->stream));
        h->parity ^= nsteps & 1;
        return LBM_OK;
    }
    int left = nsteps;
    if (h->parity == 1) {
        CUDA_TRY(launch_one(h, 1, nullptr));
        h->parity = 0;
        --left;
    }
    // graphs only on a non-default stream (capture is not allowed on the legacy stream)
    if (h->stream != nullptr && left >= kGraphSteps) {
        if (!h->graph.exec) {
            lbm_status s = capture_graph(h);
            if (s != LBM_OK) return s;
        }
        while (left >= kGraphSteps) {
            CUDA_TRY(cudaGraphLaunch(h->graph.exec, h->stream));
            left -= kGraphSteps;
        }
    }
    while (left > 0) {
        CUDA_TRY(launch_one(h, h->parity, nullptr));
        h->parity ^= 1;
        --left;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_step_timed(lbm_stefan* h, int nsteps, double* ms_kernels)
{
    if (!h || !ms_kernels) return fail(LBM_ERR_ARG, "NULL argument");
    if (h->p.lattice == LBM_D1Q3) return fail(LBM_ERR_ARG, "kernel timing covers the D2Q9 and D2Q5 steps");
    if (h->hp.method == LBM_ILFBM) return fail(LBM_ERR_STATE, "kernel timing covers the IREBM and EEBM steps");
    if (nsteps < 1) return fail(LBM_ERR_ARG, "nsteps must be >= 1");
    if (!h->ic) return fail(LBM_ERR_STATE, "set_ic must come before step_timed");
    std::vector<cudaEvent_t> ev(2 * (size_t)nsteps + 1, nullptr);
    std::vector<cudaEvent_t> fev(h->flat ? 4 * (size_t)nsteps : 0, nullptr);   // around the flat launches
    lbm_status st = LBM_OK;
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < ev.size() && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    for (size_t k = 0; k < fev.size() && e == cudaSuccess; ++k) e = cudaEventCreate(&fev[k]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], h->stream);
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        StepArgs a = single_args(h, h->parity, nullptr);
        const bool flat = h->flat && h->withhold_load < 0;
        if (h->p.lattice == LBM_D2Q5) {
            e = lbm::launch_d2q5_step(h->precision, a, h->stream);
        } else if (flat) {
            e = launch_flat(h, a, false, &fev[4 * (size_t)k]);
        } else if (h->use_tma) {
            e = lbm::launch_d2q9_tma(a, h->tma, h->stream);
        } else {
            const int grid = (h->hp.ntiles + lbm::kWarpsPerBlock - 1) / lbm::kWarpsPerBlock;
            e = lbm::launch_d2q9_step(h->precision, a, grid, h->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * k + 1], h->stream);
        if (e == cudaSuccess)
            e = flat ? launch_flat_final_jobs(h, a)
                     : lbm::launch_newton_jobs(h->precision, h->hp.q,
                                               job_args(h->dprob, 1, h->parity, nullptr, h->dstats, h->dticket,
                                                        h->djobs, h->djob_count),
                                               h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * k + 2], h->stream);
        h->parity ^= 1;
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        float a = 0.f, b = 0.f;
        e = cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[2 * k + 1], ev[2 * k + 2]);
        t0 += a;
        t1 += b;
        if (!fev.empty() && e == cudaSuccess) {
            float c = 0.f, d = 0.f;
            e = cudaEventElapsedTime(&c, fev[4 * (size_t)k], fev[4 * (size_t)k + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&d, fev[4 * (size_t)k + 2], fev[4 * (size_t)k + 3]);
            t2 += (double)c + d;
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    for (cudaEvent_t x : fev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "CUDA error: %s", cudaGetErrorString(e));
    ms_kernels[0] = t0 / nsteps;
    ms_kernels[1] = t1 / nsteps;
    ms_kernels[2] = t2 / nsteps;
    return st;
}

extern "C" lbm_status lbm_stefan_step_record(lbm_stefan* h, int nsteps, double* traj)
{
    NvtxRange r("lbm_stefan_step_record (recompute)");
    if (!h || (!traj && nsteps > 0)) return fail(LBM_ERR_ARG, "NULL argument");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (!h->ic) return fail(LBM_ERR_STATE, "set_ic must come before step_record");
    if (h->hp.method == LBM_ILFBM) return fail(LBM_ERR_STATE, "step_record records the IREBM and EEBM steps");
    const long long plane = (long long)h->hp.ny * h->hp.pitch;
    if (h->p.lattice == LBM_D1Q3 && lbm::d1q3_fused_fits(h->precision, h->hp.nx)) {
        StepArgs a = single_args(h, h->parity, nullptr);
        CUDA_TRY(lbm::launch_d1q3_fused(h->precision, a, h->hp, nsteps, h->parity, traj, h->stream));
        h->parity ^= nsteps & 1;
        return LBM_OK;
    }
    for (int k = 0; k < nsteps; ++k) {
        CUDA_TRY(launch_one(h, h->parity, traj + k * plane));
        h->parity ^= 1;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_sync(lbm_stefan* h)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return check_stats_error(h, nullptr);
}

extern "C" lbm_status lbm_stefan_get_fields(lbm_stefan* h, double* theta, double* phi, double* H, int on_device)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (!h->ic) return fail(LBM_ERR_STATE, "set_ic must come before get_fields");
    const size_t n = (size_t)h->hp.nx * h->hp.ny;
    if (on_device) {
        CUDA_TRY(lbm::launch_fields(h->precision, h->dprob, h->hp, h->parity, theta, phi, H, nullptr, h->stream));
    } else {
        double* d[3] = {theta ? h->dscratch : nullptr, phi ? h->dscratch + n : nullptr, H ? h->dscratch + 2 * n : nullptr};
        CUDA_TRY(lbm::launch_fields(h->precision, h->dprob, h->hp, h->parity, d[0], d[1], d[2], nullptr, h->stream));
        double* hst[3] = {theta, phi, H};
        for (int k = 0; k < 3; ++k)
            if (hst[k]) CUDA_TRY(cudaMemcpyAsync(hst[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    return check_stats_error(h, nullptr);
}

extern "C" lbm_status lbm_stefan_front_position(lbm_stefan* h, int wall, double* first_zero, double* integrated,
                                                double* line_first_zero, double* line_integrated)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (wall < 0 || wall > 3) return fail(LBM_ERR_ARG, "wall must be 0..3");
    if (h->p.lattice == LBM_D1Q3 && wall > 1) return fail(LBM_ERR_ARG, "D1Q3 has only the W and E walls");
    if (!h->ic) return fail(LBM_ERR_STATE, "set_ic must come before front_position");
    const int nlines = wall <= 1 ? h->hp.ny : h->hp.nx;
    CUDA_TRY(lbm::launch_front(h->precision, h->dprob, h->hp, h->parity, wall, h->dscratch, h->stream));
    std::vector<double> out(2 * (size_t)nlines);
    CUDA_TRY(cudaMemcpyAsync(out.data(), h->dscratch, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nlines; ++k) {
        a += out[k];
        b += out[nlines + k];
    }
    if (first_zero) *first_zero = a / nlines;
    if (integrated) *integrated = b / nlines;
    if (line_first_zero) std::memcpy(line_first_zero, out.data(), sizeof(double) * nlines);
    if (line_integrated) std::memcpy(line_integrated, out.data() + nlines, sizeof(double) * nlines);
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_get_stats(lbm_stefan* h, lbm_stefan_stats* out)
{
    if (!h || !out) return fail(LBM_ERR_ARG, "NULL argument");
    DevStats st;
    lbm_status s = check_stats_error(h, &st);
    out->energy = st.energy;
    out->energy_prev = st.energy_prev;
    out->flux = st.flux;
    out->imbalance = st.imbalance;
    out->imbalance_max = st.imbalance_max;
    out->steps = st.steps;
    out->newton_nodes = st.newton_nodes;
    out->newton_max_iter = st.newton_max_iter;
    out->error = st.error;
    out->newton_iters = st.newton_iters;
    return s;
}

extern "C" lbm_status lbm_stefan_set_wait_test(lbm_stefan* h, double wait_limit_s, int withhold_load)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (!(wait_limit_s > 0.0) || !(wait_limit_s <= 60.0)) return fail(LBM_ERR_ARG, "wait_limit_s must be in (0, 60]");
    if (withhold_load < -1 || withhold_load > 2) return fail(LBM_ERR_ARG, "withhold_load must be -1, 0, 1 or 2");
    h->tma.wait_ns = (long long)(wait_limit_s * 1e9);
    h->tma.withhold_load = withhold_load;
    h->withhold_load = withhold_load;
    h->graph.reset();   // captured launches carry the old values
    h->reset_seg_graphs();
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_layout(lbm_stefan* h, size_t* state_bytes, int* row_stride)
{
    if (!h) return fail(LBM_ERR_ARG, "NULL handle");
    if (state_bytes) *state_bytes = h->state_bytes;
    if (row_stride) *row_stride = h->hp.pitch;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_get_state(lbm_stefan* h, void* buf, int on_device)
{
    NvtxRange r("lbm_stefan_get_state (checkpoint)");
    if (!h || !buf) return fail(LBM_ERR_ARG, "NULL argument");
    if (!h->ic) return fail(LBM_ERR_STATE, "no state yet");
    CUDA_TRY(cudaMemcpyAsync(buf, h->hp.state[h->parity], h->state_bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_set_state(lbm_stefan* h, const void* buf, int on_device)
{
    NvtxRange r("lbm_stefan_set_state (restore)");
    if (!h || !buf) return fail(LBM_ERR_ARG, "NULL argument");
    CUDA_TRY(cudaMemcpyAsync(h->hp.state[0], buf, h->state_bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    // both buffers carry the state's shift
    CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(h->hp.state[1]) + h->hp.tail_off,
                             static_cast<const char*>(h->hp.state[0]) + h->hp.tail_off, kStateTail,
                             cudaMemcpyDeviceToDevice, h->stream));
    // the energy of a loaded state is not known until the next step publishes one
    CUDA_TRY(cudaMemsetAsync(&h->dstats->have_energy, 0, sizeof(int), h->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->parity = 0;
    h->ic = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_theta_plane(lbm_stefan* h, double* plane)
{
    if (!h || !plane) return fail(LBM_ERR_ARG, "NULL argument");
    if (!h->ic) return fail(LBM_ERR_STATE, "no state yet");
    CUDA_TRY(lbm::launch_fields(h->precision, h->dprob, h->hp, h->parity, nullptr, nullptr, nullptr, plane, h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_adjoint_seed(lbm_stefan* h, const double* theta_T, const double* phi_target,
                                              void* adj, double* loss)
{
    if (h && h->p.lattice == LBM_D2Q5) return fail(LBM_ERR_ARG, "the adjoint covers D1Q3 and D2Q9");
    if (h && h->hp.method != LBM_IREBM) return fail(LBM_ERR_STATE, "the adjoint is that of the IREBM step");
    if (!h || !theta_T || !phi_target || !adj) return fail(LBM_ERR_ARG, "NULL argument");
    CUDA_TRY(cudaMemsetAsync(&h->dstats->g_wall, 0, sizeof(lbm::Acc128) * 6, h->stream));
    CUDA_TRY(lbm::launch_adj_seed(h->precision, h->dprob, h->hp, theta_T, phi_target, adj, h->dstats, h->stream));
    if (loss) {
        DevStats st;
        lbm_status s = check_stats_error(h, &st);
        *loss = acc_host(st.loss);
        return s;
    }
    return LBM_OK;
}

static lbm::AdjArgs adj_args(lbm_stefan* h, const double* theta_t, const double* theta_t1, const void* adj_in,
                             void* adj_out)
{
    lbm::AdjArgs a;
    a.pb = h->hp;
    a.theta_t = theta_t;
    a.theta_t1 = theta_t1;
    a.adj_in = adj_in;
    a.adj_out = adj_out;
    a.stats = h->dstats;
    lbm::AdjConst& c = a.c;
    c.omc = 1.0 - h->hp.omega;
    c.om = h->hp.omega;
    c.inv_delta = h->hp.inv_delta;
    c.inv_ste = h->hp.inv_ste;
    c.thr = h->hp.sat;
    c.omc_f = (float)c.omc;
    c.om_f = (float)c.om;
    c.inv_delta_f = (float)c.inv_delta;
    c.inv_ste_f = (float)c.inv_ste;
    c.inv_ste2_f = (float)(c.inv_ste * c.inv_ste);
    c.thr_f = (float)c.thr;
    a.tile_h = h->adj_tile_h;
    a.ntiles = h->hp.nseg * ((h->hp.ny + a.tile_h - 1) / a.tile_h);
    const size_t pb = (size_t)h->hp.plane * h->elem;
    for (int i = 0; i < 9; ++i) {
        a.in_plane[i] = i < h->hp.q ? static_cast<const char*>(adj_in) + i * pb : nullptr;
        a.out_plane[i] = i < h->hp.q ? static_cast<char*>(adj_out) + i * pb : nullptr;
    }
    return a;
}

extern "C" lbm_status lbm_stefan_adjoint_step(lbm_stefan* h, const double* theta_t, const double* theta_t1,
                                              const void* adj_in, void* adj_out)
{
    if (h && h->p.lattice == LBM_D2Q5) return fail(LBM_ERR_ARG, "the adjoint covers D1Q3 and D2Q9");
    if (h && h->hp.method != LBM_IREBM) return fail(LBM_ERR_STATE, "the adjoint is that of the IREBM step");
    if (!h || !theta_t || !theta_t1 || !adj_in || !adj_out) return fail(LBM_ERR_ARG, "NULL argument");
    if (adj_in == adj_out) return fail(LBM_ERR_ARG, "adj_in and adj_out must differ");
    CUDA_TRY(lbm::launch_adj_step(h->precision, adj_args(h, theta_t, theta_t1, adj_in, adj_out), h->hp, h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_adjoint_run(lbm_stefan* h, int nsteps, const double* theta_traj, void* adj,
                                             void* adj_other, int* result_index)
{
    NvtxRange r("lbm_stefan_adjoint_run");
    if (h && h->p.lattice == LBM_D2Q5) return fail(LBM_ERR_ARG, "the adjoint covers D1Q3 and D2Q9");
    if (h && h->hp.method != LBM_IREBM) return fail(LBM_ERR_STATE, "the adjoint is that of the IREBM step");
    if (!h || !adj || !adj_other || !result_index || (!theta_traj && nsteps > 0))
        return fail(LBM_ERR_ARG, "NULL argument");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (adj == adj_other) return fail(LBM_ERR_ARG, "adj and adj_other must differ");
    const long long plane = (long long)h->hp.ny * h->hp.pitch;
    void* buf[2] = {adj, adj_other};
    int cur = 0;
    for (int s = nsteps - 1; s >= 0; --s) {
        CUDA_TRY(lbm::launch_adj_step(h->precision,
                                      adj_args(h, theta_traj + s * plane, theta_traj + (s + 1) * plane, buf[cur],
                                               buf[cur ^ 1]),
                                      h->hp, h->stream));
        cur ^= 1;
    }
    *result_index = cur;
    return LBM_OK;
}

// The launches of one backward segment after the checkpoint is loaded: theta(t0)
// into traj[0], nsteps recorded steps, nsteps reverse steps.
static cudaError_t segment_launches(lbm_stefan* h, int nsteps, double* traj, void* a, void* b, int parity0)
{
    const long long plane = (long long)h->hp.ny * h->hp.pitch;
    cudaError_t e = lbm::launch_fields(h->precision, h->dprob, h->hp, parity0, nullptr, nullptr, nullptr, traj,
                                       h->stream);
    int par = parity0;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        e = launch_one(h, par, traj + (k + 1) * plane);
        par ^= 1;
    }
    void* buf[2] = {a, b};
    int cur = 0;
    for (int s = nsteps - 1; s >= 0 && e == cudaSuccess; --s) {
        e = lbm::launch_adj_step(h->precision, adj_args(h, traj + s * plane, traj + (s + 1) * plane, buf[cur], buf[cur ^ 1]),
                                 h->hp, h->stream);
        cur ^= 1;
    }
    return e;
}

extern "C" lbm_status lbm_stefan_adjoint_segment(lbm_stefan* h, const void* checkpoint, int nsteps, double* theta_traj,
                                                 void* adj, void* adj_other, int* result_index)
{
    NvtxRange r("lbm_stefan_adjoint_segment (restore, recompute, reverse steps)");
    if (h && h->p.lattice != LBM_D2Q9) return fail(LBM_ERR_ARG, "adjoint_segment covers D2Q9 (D1Q3: adjoint_run)");
    if (h && h->hp.method != LBM_IREBM) return fail(LBM_ERR_STATE, "the adjoint is that of the IREBM step");
    if (!h || !checkpoint || !theta_traj || !adj || !adj_other || !result_index) return fail(LBM_ERR_ARG, "NULL argument");
    if (nsteps < 1) return fail(LBM_ERR_ARG, "nsteps must be >= 1");
    if (adj == adj_other) return fail(LBM_ERR_ARG, "adj and adj_other must differ");
    // reload the checkpoint into state[0]
    CUDA_TRY(cudaMemcpyAsync(h->hp.state[0], checkpoint, h->state_bytes, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(h->hp.state[1]) + h->hp.tail_off,
                             static_cast<const char*>(h->hp.state[0]) + h->hp.tail_off, kStateTail,
                             cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemsetAsync(&h->dstats->have_energy, 0, sizeof(int), h->stream));
    h->parity = 0;
    h->ic = true;
    cudaGraphExec_t exec = nullptr;
    for (auto& g : h->seg_graphs)
        if (g.n == nsteps && g.traj == theta_traj && g.a == adj && g.b == adj_other) exec = g.exec;
    if (!exec && h->stream != nullptr) {
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = segment_launches(h, nsteps, theta_traj, adj, adj_other, 0);
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
        if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || e2 != cudaSuccess || !exec)
            return fail(LBM_ERR_CUDA, "segment capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        if (h->seg_graphs.size() >= 8) h->reset_seg_graphs();
        h->seg_graphs.push_back({nsteps, theta_traj, adj, adj_other, exec});
    }
    if (exec) CUDA_TRY(cudaGraphLaunch(exec, h->stream));
    else CUDA_TRY(segment_launches(h, nsteps, theta_traj, adj, adj_other, 0));
    h->parity = nsteps & 1;
    *result_index = nsteps & 1;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_adjoint_finish(lbm_stefan* h, const void* adj0, double* g_theta0, int on_device,
                                                double* g_wall, double* g_ste)
{
    if (h && h->p.lattice == LBM_D2Q5) return fail(LBM_ERR_ARG, "the adjoint covers D1Q3 and D2Q9");
    if (!h || !adj0) return fail(LBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->hp.nx * h->hp.ny;
    double* dst = (g_theta0 && on_device) ? g_theta0 : h->dscratch;
    CUDA_TRY(lbm::launch_adj_finish(h->precision, h->dprob, h->hp, adj0, dst, h->dstats, h->stream));
    if (g_theta0 && !on_device)
        CUDA_TRY(cudaMemcpyAsync(g_theta0, h->dscratch, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DevStats st;
    lbm_status s = check_stats_error(h, &st);
    if (g_wall)
        for (int k = 0; k < 4; ++k) g_wall[k] = h->hp.wall_kind[k] == LBM_DIRICHLET ? acc_host(st.g_wall[k]) : 0.0;
    if (g_ste) *g_ste = acc_host(st.g_ste);
    return s;
}

extern "C" void lbm_stefan_destroy(lbm_stefan* h)
{
    if (!h) return;
    h->graph.reset();
    h->reset_seg_graphs();
    cudaFree(h->hp.state[0]);
    cudaFree(h->hp.state[1]);
    cudaFree(h->dprob);
    cudaFree(h->dstats);
    cudaFree(h->dticket);
    cudaFree(h->dscratch);
    cudaFree(h->djobs);
    cudaFree(h->djob_count);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_half) cudaEventDestroy(h->ev_half);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_walls) cudaEventDestroy(h->ev_walls);
    if (h->side) cudaStreamDestroy(h->side);
    cudaFree(h->dilf);
    cudaFree(h->dilf_scratch);
    delete h;
}

extern "C" const char* lbm_stefan_last_error(void) { return g_err; }

// ------------------------------------------------------------------ batches

// Descriptors of every problem's two state buffers for the TMA kernel; false
// leaves the batch on the warp-tile kernel.
// Flat-kernel tables: every problem's 128-column strips in 8-row tiles
// (strips fastest, then bands), and its S and N rows; schedule 1 puts the
// largest problems first.
static lbm_status batch_build_flat_tables(lbm_stefan_batch* b, int schedule)
{
    std::vector<int> order(b->count);
    for (int k = 0; k < b->count; ++k) order[k] = k;
    if (schedule == 1)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (long long)b->hp[x].nx * b->hp[x].ny > (long long)b->hp[y].nx * b->hp[y].ny;
        });
    // every problem's left-half tiles (strips below max(1, nsegs / 2)), then the
    // right-half tiles: the split step solves the first group's Newton nodes
    // beside the second group's streaming
    std::vector<int4> tiles;
    std::vector<int2> rows, crows;
    for (int side = 0; side < 2; ++side) {
        for (int k : order) {
            const Problem& pb = b->hp[k];
            const int nsegs = pb.pitch / lbm::kTmaW;
            const int half = std::max(1, nsegs / 2);
            if (pb.ny > 2)
                for (int y0 = 0; y0 < pb.ny - 1; y0 += 8)
                    for (int seg = side ? half : 0; seg < (side ? nsegs : half); ++seg)
                        tiles.push_back(make_int4(k, seg, y0, 0));
        }
        if (side == 0) b->nftiles_left = (int)tiles.size();
    }
    for (int k : order) {
        const Problem& pb = b->hp[k];
        const int nsegs = pb.pitch / lbm::kTmaW;
        if (pb.ny > 2)
            for (int y0 = 1; y0 < pb.ny - 1; y0 += 32) crows.push_back(make_int2(k, y0));
        for (int seg = 0; seg < nsegs; ++seg) {
            rows.push_back(make_int2(k, 2 * seg));
            rows.push_back(make_int2(k, 2 * seg + 1));
        }
    }
    cudaFree(b->dftiles);
    cudaFree(b->dwrows);
    cudaFree(b->dcrows);
    b->dftiles = nullptr;
    b->dwrows = nullptr;
    b->dcrows = nullptr;
    CUDA_TRY(cudaMalloc(&b->dftiles, sizeof(int4) * std::max<size_t>(1, tiles.size())));
    CUDA_TRY(cudaMemcpy(b->dftiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&b->dwrows, sizeof(int2) * rows.size()));
    CUDA_TRY(cudaMemcpy(b->dwrows, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&b->dcrows, sizeof(int2) * std::max<size_t>(1, crows.size())));
    CUDA_TRY(cudaMemcpy(b->dcrows, crows.data(), sizeof(int2) * crows.size(), cudaMemcpyHostToDevice));
    b->nftiles = (int)tiles.size();
    b->nwrows = (int)rows.size();
    b->ncblocks = (int)crows.size();
    return LBM_OK;
}

static lbm_status batch_build_schedule(lbm_stefan_batch* b, int tile_h, int schedule)
{
    const int segw = lbm::d2q9_segment_width(b->precision);
    int total = 0;
    for (auto& pb : b->hp) {
        pb.tile_h = tile_h;
        pb.nstrip = (pb.ny + tile_h - 1) / tile_h;
        pb.nseg = pb.pitch / segw;
        pb.ntiles = pb.nseg * pb.nstrip;
        pb.tile0 = total;
        total += pb.ntiles;
    }
    std::vector<int2> sched;
    sched.reserve(total);
    for (int k = 0; k < b->count; ++k)
        for (int t = 0; t < b->hp[k].ntiles; ++t) sched.push_back(make_int2(k, t));
    if (schedule == 1) {
        // longest tiles first: a ragged last strip is shorter; ties keep problem order
        std::stable_sort(sched.begin(), sched.end(), [&](const int2& a, const int2& c) {
            auto rows = [&](const int2& s) {
                const Problem& pb = b->hp[s.x];
                const int strip = s.y / pb.nseg;
                return std::min(pb.ny, (strip + 1) * pb.tile_h) - strip * pb.tile_h;
            };
            return rows(a) > rows(c);
        });
    }
    if (b->dsched) cudaFree(b->dsched);
    b->dsched = nullptr;
    CUDA_TRY(cudaMalloc(&b->dsched, sizeof(int2) * sched.size()));
    CUDA_TRY(cudaMemcpy(b->dsched, sched.data(), sizeof(int2) * sched.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b->dprobs, b->hp.data(), sizeof(Problem) * b->count, cudaMemcpyHostToDevice));
    CUDA_TRY(lbm::launch_wall_constants(b->dprobs, b->count, nullptr));
    CUDA_TRY(cudaDeviceSynchronize());
    b->nslots = total;
    b->tile_h = b->use_flat ? 8 : tile_h;
    b->schedule = schedule;
    b->graph.reset();
    if (b->use_flat) {
        lbm_status s = batch_build_flat_tables(b, schedule);
        if (s != LBM_OK) return s;
    }
    // persistent grid: as many blocks as fit on the GPU at once
    int dev = 0, sms = 0, per_sm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    per_sm = lbm::d2q9_blocks_per_sm(b->precision);
    b->grid = std::max(1, std::min(sms * per_sm, (total + lbm::kWarpsPerBlock - 1) / lbm::kWarpsPerBlock));
    return LBM_OK;
}

static cudaError_t batch_launch_one(lbm_stefan_batch* b, int parity)
{
    StepArgs a;
    a.probs = b->dprobs;
    a.nprob = b->count;
    a.schedule = b->dsched;
    a.nslots = b->nslots;
    a.parity = parity;
    a.rec = nullptr;
    a.stats = b->dstats;
    a.ticket = b->dticket;
    a.jobs = b->djobs;
    a.job_count = b->djob_count;
    cudaError_t e;
    if (b->use_flat && b->side) {
        // as the single problem's split step: the wall kernels, then the Newton
        // solves of the wall nodes and the left halves (list A, shared cursor)
        // on the side stream beside the right halves'
        // streaming; then a full job launch takes the rest of list A and list B
        int least = 0, prio = 0;
        const int sms = device_sms();
        e = sms > 0 ? cudaDeviceGetStreamPriorityRange(&least, &prio) : cudaErrorInvalidDevice;
        a.ftiles = b->dftiles;
        a.wrows = b->dwrows;
        a.nwrows = b->nwrows;
        a.crows = b->dcrows;
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
        if (e == cudaSuccess) e = lbm::launch_d2q9_flat(a, 0, b->nwrows, b->ncblocks, 0, b->side);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_walls, b->side);
        if (e == cudaSuccess) e = lbm::launch_d2q9_flat(a, b->nftiles_left, 0, 0, 0, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_half, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_half, 0);
        if (e != cudaSuccess) return e;
        const int gb = 2 * sms;
        const lbm::JobArgs ja = split_jobs_first(b->dprobs, b->count, parity, nullptr, b->dstats, b->dticket, b->djobs,
                                                 b->djob_count, sms + gb);
        e = lbm::launch_newton_jobs(b->precision, 9, ja, b->side, sms, prio, true);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->side);
        if (e != cudaSuccess) return e;
        StepArgs ab = a;
        ab.ftiles = b->dftiles + b->nftiles_left;
        ab.jobs = b->djobs + b->total_nodes;
        ab.job_count = b->djob_count + 1;
        e = lbm::launch_d2q9_flat(ab, b->nftiles - b->nftiles_left, 0, 0, 0, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_walls, 0);   // list A's wall nodes are in
        if (e == cudaSuccess)
            e = lbm::launch_newton_jobs(b->precision, 9, split_jobs_last(ja, ab.jobs), b->stream, gb);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
        return e;
    }
    if (b->use_flat) {
        a.ftiles = b->dftiles;
        a.wrows = b->dwrows;
        a.nwrows = b->nwrows;
        a.crows = b->dcrows;
        e = lbm::launch_d2q9_flat(a, b->nftiles, b->nwrows, b->ncblocks, 0, b->stream);
    } else {
        e = lbm::launch_d2q9_step(b->precision, a, b->grid, b->stream);
    }
    if (e != cudaSuccess) return e;
    return lbm::launch_newton_jobs(b->precision, 9,
                                   job_args(b->dprobs, b->count, parity, nullptr, b->dstats, b->dticket, b->djobs,
                                            b->djob_count),
                                   b->stream);
}

extern "C" lbm_status lbm_stefan_batch_create(int count, const lbm_stefan_problem* probs, int precision,
                                              double newton_tol, int newton_max_iter, void* cuda_stream,
                                              lbm_stefan_batch** out)
{
    if (!out || !probs || count < 1) return fail(LBM_ERR_ARG, "need count >= 1 problems");
    *out = nullptr;
    if (precision != LBM_FP32 && precision != LBM_FP64) return fail(LBM_ERR_ARG, "precision must be FP64 or FP32");
    lbm_stefan_batch* b = new lbm_stefan_batch();
    b->count = count;
    b->precision = precision;
    b->elem = precision == LBM_FP32 ? 4 : 8;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    const int segw = lbm::d2q9_segment_width(precision);
    size_t total = 0;
    size_t maxn = 0;
    size_t total_nodes = 0;
    b->hp.resize(count);
    b->state_bytes.resize(count);
    for (int k = 0; k < count; ++k) {
        const lbm_stefan_problem& p = probs[k];
        lbm_status s = validate_common(p.nx, p.ny, p.tau, p.delta, p.ste, newton_tol, newton_max_iter);
        if (s == LBM_OK && p.ny < 2) s = fail(LBM_ERR_ARG, "problem %d: ny must be >= 2", k);
        for (int w = 0; w < 4 && s == LBM_OK; ++w)
            if ((p.wall_kind[w] != 0 && p.wall_kind[w] != 1) || !std::isfinite(p.wall_theta[w]))
                s = fail(LBM_ERR_ARG, "problem %d: bad wall %d", k, w);
        if (s != LBM_OK) {
            delete b;
            return s;
        }
        Problem& pb = b->hp[k];
        fill_problem(pb, 9, p.nx, p.ny, state_pitch(LBM_D2Q9, precision, p.nx), p.tau, p.delta, p.ste, newton_tol,
                     newton_max_iter, LBM_BB_MIRROR, 16, segw, precision);
        for (int w = 0; w < 4; ++w) {
            pb.wall_kind[w] = p.wall_kind[w];
            pb.wall_theta[w] = p.wall_theta[w];
        }
        pb.stats = k;
        b->state_bytes[k] = (size_t)pb.tail_off + kStateTail;
        total += 2 * ((b->state_bytes[k] + 255) / 256 * 256);
        maxn = std::max(maxn, (size_t)p.nx * p.ny);
        total_nodes += (size_t)p.nx * p.ny;
    }
    cudaError_t e = cudaMalloc(&b->arena, total);
    if (e == cudaSuccess) e = cudaMemset(b->arena, 0, total);
    if (e == cudaSuccess) e = cudaMalloc(&b->dprobs, sizeof(Problem) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->dstats, sizeof(DevStats) * count);
    if (e == cudaSuccess) e = cudaMemset(b->dstats, 0, sizeof(DevStats) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->dticket, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(b->dticket, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->dscratch, sizeof(double) * maxn);
    // FP32 on a stream of its own: the split step, two job lists of total_nodes each
    const bool split = precision == LBM_FP32 && LBM_SPLIT && b->stream != nullptr;
    if (e == cudaSuccess && split) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_half, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_walls, cudaEventDisableTiming);
    }
    b->total_nodes = total_nodes;
    if (e == cudaSuccess) e = cudaMalloc(&b->djobs, sizeof(lbm::NewtonJob) * total_nodes * (split ? 2 : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->djob_count, 3 * sizeof(unsigned int));   // lists A, B; cursor of A
    if (e == cudaSuccess) e = cudaMemset(b->djob_count, 0, 3 * sizeof(unsigned int));
    if (e != cudaSuccess) {
        lbm_stefan_batch_destroy(b);
        return fail(LBM_ERR_CUDA, "batch allocation failed: %s", cudaGetErrorString(e));
    }
    b->arena_bytes = total;
    b->scratch_elems = maxn;
    char* base = static_cast<char*>(b->arena);
    for (int k = 0; k < count; ++k) {
        const size_t sz = (b->state_bytes[k] + 255) / 256 * 256;
        b->hp[k].state[0] = base;
        b->hp[k].state[1] = base + sz;
        base += 2 * sz;
    }
    b->use_flat = precision == LBM_FP32;
    cudaGetLastError();
    lbm_status s = batch_build_schedule(b, 16, 1);
    if (s != LBM_OK) {
        lbm_stefan_batch_destroy(b);
        return s;
    }
    *out = b;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_batch_set_ic(lbm_stefan_batch* b, int k, const double* theta0, int on_device)
{
    if (!b || !theta0) return fail(LBM_ERR_ARG, "NULL argument");
    if (k < 0 || k >= b->count) return fail(LBM_ERR_ARG, "problem index out of range");
    if (b->parity != 0) return fail(LBM_ERR_STATE, "set_ic on a batch needs an even step count so far");
    const Problem& hp = b->hp[k];
    const size_t n = (size_t)hp.nx * hp.ny;
    const double* src = theta0;
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(b->dscratch, theta0, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        src = b->dscratch;
    }
    CUDA_TRY(cudaMemsetAsync(b->dstats + k, 0, sizeof(DevStats), b->stream));
    CUDA_TRY(lbm::launch_init_state(b->precision, b->dprobs + k, hp, src, 0, b->dstats + k, b->stream));
    CUDA_TRY(lbm::launch_finalize_init(b->dstats + k, b->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

static lbm_status batch_capture(lbm_stefan_batch* b)
{
    b->graph.reset();
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = batch_launch_one(b, k & 1);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(LBM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph.exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    b->graph.steps = kGraphSteps;
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_batch_step(lbm_stefan_batch* b, int nsteps)
{
    NvtxRange r("lbm_stefan_batch_step");
    if (!b) return fail(LBM_ERR_ARG, "NULL handle");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
    int left = nsteps;
    if (b->parity == 1 && left > 0) {
        CUDA_TRY(batch_launch_one(b, 1));
        b->parity = 0;
        --left;
    }
    if (b->stream != nullptr && left >= kGraphSteps) {
        if (!b->graph.exec) {
            lbm_status s = batch_capture(b);
            if (s != LBM_OK) return s;
        }
        while (left >= kGraphSteps) {
            CUDA_TRY(cudaGraphLaunch(b->graph.exec, b->stream));
            left -= kGraphSteps;
        }
    }
    while (left > 0) {
        CUDA_TRY(batch_launch_one(b, b->parity));
        b->parity ^= 1;
        --left;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_batch_get_fields(lbm_stefan_batch* b, int k, double* theta, int on_device)
{
    if (!b || !theta) return fail(LBM_ERR_ARG, "NULL argument");
    if (k < 0 || k >= b->count) return fail(LBM_ERR_ARG, "problem index out of range");
    const Problem& hp = b->hp[k];
    const size_t n = (size_t)hp.nx * hp.ny;
    double* dst = on_device ? theta : b->dscratch;
    CUDA_TRY(lbm::launch_fields(b->precision, b->dprobs + k, hp, b->parity, dst, nullptr, nullptr, nullptr, b->stream));
    if (!on_device) CUDA_TRY(cudaMemcpyAsync(theta, b->dscratch, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    DevStats st;
    CUDA_TRY(cudaMemcpy(&st, b->dstats + k, sizeof st, cudaMemcpyDeviceToHost));
    if (st.error) return fail((lbm_status)st.error, "device reported error %d in problem %d", st.error, k);
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_batch_get_stats(lbm_stefan_batch* b, int k, lbm_stefan_stats* out)
{
    if (!b || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (k < 0 || k >= b->count) return fail(LBM_ERR_ARG, "problem index out of range");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    DevStats st;
    CUDA_TRY(cudaMemcpy(&st, b->dstats + k, sizeof st, cudaMemcpyDeviceToHost));
    out->energy = st.energy;
    out->energy_prev = st.energy_prev;
    out->flux = st.flux;
    out->imbalance = st.imbalance;
    out->imbalance_max = st.imbalance_max;
    out->steps = st.steps;
    out->newton_nodes = st.newton_nodes;
    out->newton_max_iter = st.newton_max_iter;
    out->error = st.error;
    out->newton_iters = st.newton_iters;
    if (st.error) return fail((lbm_status)st.error, "device reported error %d in problem %d", st.error, k);
    return LBM_OK;
}

extern "C" lbm_status lbm_stefan_batch_set_schedule(lbm_stefan_batch* b, int tile_h, int schedule)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL handle");
    if (tile_h < 1 || tile_h > 4096) return fail(LBM_ERR_ARG, "tile_h must be in 1..4096");
    if (schedule != 0 && schedule != 1) return fail(LBM_ERR_ARG, "schedule must be 0 or 1");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return batch_build_schedule(b, tile_h, schedule);
}

extern "C" lbm_status lbm_stefan_batch_autotune(lbm_stefan_batch* b, int trial_steps, int* chosen_tile_h)
{
    if (!b) return fail(LBM_ERR_ARG, "NULL handle");
    if (trial_steps < 1) return fail(LBM_ERR_ARG, "trial_steps must be >= 1");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    // save the current state and statistics, try each candidate, restore
    void* save = nullptr;
    DevStats* save_st = nullptr;
    CUDA_TRY(cudaMalloc(&save, b->arena_bytes));
    cudaError_t e = cudaMalloc(&save_st, sizeof(DevStats) * b->count);
    if (e != cudaSuccess) {
        cudaFree(save);
        return fail(LBM_ERR_CUDA, "autotune allocation failed: %s", cudaGetErrorString(e));
    }
    cudaMemcpyAsync(save, b->arena, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(save_st, b->dstats, sizeof(DevStats) * b->count, cudaMemcpyDeviceToDevice, b->stream);
    const int saved_parity = b->parity;
    const int cands_h[] = {8, 16, 32, 64};   // rows per tile
    const int cands_s[] = {1, 0};
    float best = 1e30f;
    int best_h = b->tile_h, best_s = b->schedule;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    lbm_status st = LBM_OK;
    // the flat FP32 kernels have fixed 8-row tiles: only the order is tuned
    for (int ci = 0; ci < (b->use_flat ? 1 : 4); ++ci) {
        const int hs = cands_h[ci];
        for (int sc : cands_s) {
            st = batch_build_schedule(b, hs, sc);
            if (st != LBM_OK) break;
            // one untimed warm-up step, then the timed trial
            if (batch_launch_one(b, b->parity) != cudaSuccess) { st = fail(LBM_ERR_CUDA, "autotune launch failed"); break; }
            b->parity ^= 1;
            cudaEventRecord(e0, b->stream);
            for (int k = 0; k < trial_steps; ++k) {
                if (batch_launch_one(b, b->parity) != cudaSuccess) { st = fail(LBM_ERR_CUDA, "autotune launch failed"); break; }
                b->parity ^= 1;
            }
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_h = hs;
                best_s = sc;
            }
            cudaMemcpyAsync(b->arena, save, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream);
            b->parity = saved_parity;
        }
        if (st != LBM_OK) break;
    }
    cudaMemcpyAsync(b->dstats, save_st, sizeof(DevStats) * b->count, cudaMemcpyDeviceToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save);
    cudaFree(save_st);
    if (st != LBM_OK) return st;
    st = batch_build_schedule(b, best_h, best_s);
    if (chosen_tile_h) *chosen_tile_h = best_h;
    return st;
}

extern "C" void lbm_stefan_batch_destroy(lbm_stefan_batch* b)
{
    if (!b) return;
    b->graph.reset();
    cudaFree(b->arena);
    cudaFree(b->dprobs);
    cudaFree(b->dstats);
    cudaFree(b->dticket);
    cudaFree(b->dsched);
    cudaFree(b->dscratch);
    cudaFree(b->djobs);
    cudaFree(b->djob_count);
    cudaFree(b->dftiles);
    cudaFree(b->dwrows);
    cudaFree(b->dcrows);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_half) cudaEventDestroy(b->ev_half);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->ev_walls) cudaEventDestroy(b->ev_walls);
    if (b->side) cudaStreamDestroy(b->side);
    delete b;
}

// ------------------------------------------------------------------ one step without allocation
//
// For callers that cannot allocate device memory when they step: code running
// under an allocator or memory budget it does not own, pre-sized real-time loops
// that must not call cudaMalloc (it can block and synchronize the device), or
// hosts whose GPU memory is handed out up front.  They own the two state buffers;
// the step's scratch (problem descriptor, statistics, counters and the list of
// nodes whose Newton solve is deferred) lives in this fixed device array.  Every
// GPU that loads the library holds it until the process exits.

namespace {

constexpr int kNoAllocMaxNodes = 1 << 18;   // 262,144 nodes (e.g. 512 x 512)

struct NoAllocScratch {
    Problem prob;
    DevStats stats;
    unsigned int ticket;
    unsigned int job_count;
    lbm::NewtonJob jobs[kNoAllocMaxNodes];
};

// about 6.3 MB
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Bytes that each call clears: the statistics, the last-block ticket and the
// job count, which lie between `stats` and `jobs`.
constexpr size_t kNoAllocClear = offsetof(NoAllocScratch, jobs) - offsetof(NoAllocScratch, stats);
static_assert(offsetof(NoAllocScratch, ticket) >= offsetof(NoAllocScratch, stats) + sizeof(DevStats) &&
                  offsetof(NoAllocScratch, job_count) + sizeof(unsigned int) <= offsetof(NoAllocScratch, jobs),
              "the counters must lie in the cleared range");

// Device address of the scratch array, resolved once per CUDA context: host
// code cannot use the array's name as a device address, and a context that is
// destroyed and created again (cudaDeviceReset) may place the array elsewhere.
std::mutex g_noalloc_mutex;
std::vector<std::pair<CUcontext, void*>> g_noalloc_addr;

PFN_cuCtxGetCurrent_v4000 ctx_getter()
{
    static const PFN_cuCtxGetCurrent_v4000 fn = []() -> PFN_cuCtxGetCurrent_v4000 {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
    }();
    return fn;
}

lbm_status noalloc_scratch(NoAllocScratch** out, cudaStream_t stream)
{
    // a query of the caller's stream makes the device's context current
    // (nothing is allocated or waited for)
    const cudaError_t q = cudaStreamQuery(stream);
    if (q != cudaSuccess && q != cudaErrorNotReady) return fail(LBM_ERR_CUDA, "cudaStreamQuery: %s", cudaGetErrorString(q));
    const PFN_cuCtxGetCurrent_v4000 get = ctx_getter();
    CUcontext ctx = nullptr;
    if (!get || get(&ctx) != CUDA_SUCCESS || !ctx) return fail(LBM_ERR_CUDA, "no current CUDA context");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    for (const auto& e : g_noalloc_addr)
        if (e.first == ctx) {
            *out = static_cast<NoAllocScratch*>(e.second);
            return LBM_OK;
        }
    void* ptr = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_addr.emplace_back(ctx, ptr);
    *out = static_cast<NoAllocScratch*>(ptr);
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_stefan_step_d2q9_noalloc(const lbm_stefan_params* p, const int* wall_kind,
                                                   const double* wall_theta, const void* state_in, void* state_out,
                                                   void* cuda_stream)
{
    if (!p || !wall_kind || !wall_theta || !state_in || !state_out) return fail(LBM_ERR_ARG, "NULL argument");
    if (state_in == state_out) return fail(LBM_ERR_ARG, "state_in and state_out must differ");
    if (p->lattice != LBM_D2Q9) return fail(LBM_ERR_ARG, "the no-allocation step is D2Q9 only");
    if (p->precision != LBM_FP64 && p->precision != LBM_FP32) return fail(LBM_ERR_ARG, "precision must be FP64 or FP32");
    if (p->bb_mode != LBM_BB_MIRROR && p->bb_mode != LBM_BB_LINK) return fail(LBM_ERR_ARG, "bb_mode must be 0 or 1");
    lbm_status s = validate_common(p->nx, p->ny, p->tau, p->delta, p->ste, p->newton_tol, p->newton_max_iter);
    if (s != LBM_OK) return s;
    if (p->ny < 2) return fail(LBM_ERR_ARG, "D2Q9 needs ny >= 2");
    if ((long long)p->nx * p->ny > kNoAllocMaxNodes)
        return fail(LBM_ERR_ARG, "no-allocation step: %d x %d = %lld nodes exceed the maximum of %d", p->nx, p->ny,
                    (long long)p->nx * p->ny, kNoAllocMaxNodes);
    for (int w = 0; w < 4; ++w)
        if ((wall_kind[w] != LBM_ADIABATIC && wall_kind[w] != LBM_DIRICHLET) || !std::isfinite(wall_theta[w]))
            return fail(LBM_ERR_ARG, "bad wall %d", w);

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    NoAllocScratch* sc = nullptr;
    s = noalloc_scratch(&sc, st);
    if (s != LBM_OK) return s;

    const int segw = lbm::d2q9_segment_width(p->precision);
    Problem hp;
    fill_problem(hp, 9, p->nx, p->ny, state_pitch(LBM_D2Q9, p->precision, p->nx), p->tau, p->delta, p->ste, p->newton_tol,
                 p->newton_max_iter, p->bb_mode, 16, segw, p->precision);
    for (int w = 0; w < 4; ++w) {
        hp.wall_kind[w] = wall_kind[w];
        hp.wall_theta[w] = wall_theta[w];
    }
    hp.state[0] = const_cast<void*>(state_in);
    hp.state[1] = state_out;
    hp.stats = 0;
    // the array keeps the previous call's contents: statistics, ticket and job
    // count must start at zero
    CUDA_TRY(cudaMemcpyAsync(&sc->prob, &hp, sizeof(Problem), cudaMemcpyHostToDevice, st));
    // the output state carries the input's shift (its tail)
    CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(state_out) + hp.tail_off,
                             static_cast<const char*>(state_in) + hp.tail_off, kStateTail, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemsetAsync(&sc->stats, 0, kNoAllocClear, st));
    CUDA_TRY(lbm::launch_wall_constants(&sc->prob, 1, st));

    StepArgs a;
    a.probs = &sc->prob;
    a.nprob = 1;
    a.schedule = nullptr;
    a.nslots = hp.ntiles;
    a.parity = 0;
    a.rec = nullptr;
    a.stats = &sc->stats;
    a.ticket = &sc->ticket;
    a.jobs = sc->jobs;
    a.job_count = &sc->job_count;
    CUDA_TRY(lbm::launch_d2q9_step(p->precision, a, (hp.ntiles + lbm::kWarpsPerBlock - 1) / lbm::kWarpsPerBlock, st));
    CUDA_TRY(lbm::launch_newton_jobs(p->precision, 9,
                                     job_args(&sc->prob, 1, 0, nullptr, &sc->stats, &sc->ticket, sc->jobs, &sc->job_count),
                                     st));
    // report a device-detected Newton failure: read the flag (this waits for the step)
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, &sc->stats.error, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (err) return fail((lbm_status)err, "device reported error %d (Newton limit or non-finite value)", err);
    return LBM_OK;
}
