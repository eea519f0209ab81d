// Fused FP32 D2Q9 IREBM step: one persistent launch per time step of
// Algorithm 3, stream + closures + moments + local Newton solve (Eq. 14) +
// source and relaxation (Eqs. 12-13), FP32 populations with the FP64 Newton.
//
// One block per SM, two warp roles.
//
// Streaming warps (kStreamWarps per block).  Every streaming warp is an
// independent worker.  A work item is a 128-column strip of one problem over
// a range of rows [ya, yb); a warp takes items in list order from a global
// counter (the list is guided self-scheduling: the items taken last are one
// or two rows, so the warps finish together) and handles four consecutive
// columns per lane.  Each streaming warp owns kFusedStages shared-memory
// slots; one slot holds one row of all nine planes, 136 columns (the strip
// plus 4 columns on each side, zero-filled by TMA outside the tensor).  Lane
// 0 issues one cp.async.bulk.tensor load per row, completing on the slot's
// mbarrier; the loads run ahead through the rows of the current item and
// into the next one.  For row y the warp reads planes 0,1,2,3,5,6 of row y
// and planes 4,7,8 of row y+1 (the pulls along -y); the pulls along +y
// (planes 2,5,6 of row y-1) and the unshifted planes 4,7,8 of row y (for
// theta = sum Omega) come from registers kept from the previous row.  Per
// four nodes a lane issues nine 128-bit and six 32-bit shared loads and nine
// 128-bit global stores.  A slot is refilled only after the values read from
// it have been used in arithmetic.
//
// Newton warps (kNewtonWarps per block, one per SM sub-partition).  A node
// outside the saturated branch is stored unrelaxed by its streaming warp and
// its (m0, theta) are appended to a queue of that warp in shared memory; each
// time 32 are queued (and once more at the end, padded), the warp writes them
// as one batch to a global array (slot from a global counter), fences, and
// appends the batch's index to the queue of block (slot mod blocks).  The
// Newton warps of each block take batches from their block's queue (a tail
// in global memory, written by other blocks; a head in shared memory) and
// solve them, one node per lane (the FP64 mixed-precision Newton of
// newton_mixed), relaxing the nodes' populations in place.  On this GPU the
// FP64 unit of a sub-partition needs tens of cycles per warp-wide FP64
// instruction, so a batch occupies a warp for thousands of cycles: dedicated
// warps keep that off the streaming warps, and the front band's FP64 work is
// spread over every SM while the streaming goes on.  Newton warps stop when
// no streaming warp of the launch is left and their queue is empty; the
// launch is cooperative (every block resident), since warps wait for others.
//
// Waits.  Every wait (row loads, queue entries, the streaming warps' end) is
// bounded in time (FusedArgs::wait_ns).  A streaming warp whose wait for a row
// load runs out records LBM_ERR_TIMEOUT, waits (bounded) for the loads it
// still has in flight and stops taking items.
#include "d2q9_row.cuh"

namespace lbm {

#ifndef LBM_FUSED_STAGES
#define LBM_FUSED_STAGES 9
#endif
#ifndef LBM_FUSED_STREAM_WARPS
#define LBM_FUSED_STREAM_WARPS 4
#endif
#ifndef LBM_FUSED_NEWTON_WARPS
#define LBM_FUSED_NEWTON_WARPS 4
#endif
constexpr int kFusedStages = LBM_FUSED_STAGES;        // row slots per streaming warp
constexpr int kStreamWarps = LBM_FUSED_STREAM_WARPS;  // streaming warps per block
constexpr int kNewtonWarps = LBM_FUSED_NEWTON_WARPS;  // Newton warps per block
constexpr int kFusedThreads = 32 * (kStreamWarps + kNewtonWarps);
constexpr int kFusedQueue = 160;                      // < 32 left over + one row (128 nodes)
constexpr int kRowBox = kTmaW + 2 * kTmaHalo;         // 136 loaded columns per plane row
constexpr int kRowSlot = (9 * kRowBox * 4 + 127) / 128 * 32;   // floats per slot (128-byte multiple)
constexpr unsigned kRowBytes = 9u * kRowBox * 4u;               // bytes one row load delivers

struct alignas(128) StreamWarp {
    float ring[kFusedStages][kRowSlot];
    NewtonJob queue[kFusedQueue];
    unsigned long long full[kFusedStages];
};
constexpr int kFusedSmem = kStreamWarps * (int)sizeof(StreamWarp);

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase `parity` of a row-load mbarrier, at most limit_ns.
__device__ __forceinline__ bool mbar_wait_ns(unsigned long long* b, unsigned parity, long long limit_ns)
{
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(b, parity)) return true;
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    }
}

__device__ __forceinline__ void ld4(const float* p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

// Queue of a warp's deferred Newton nodes (the sink of row_update).  n is
// the same in every lane.
struct WarpQueueSink {
    NewtonJob* q;
    int n;
    __device__ __forceinline__ unsigned reserve(unsigned total, int) { const unsigned b = (unsigned)n; n += (int)total; return b; }
    __device__ __forceinline__ void put(unsigned slot, const NewtonJob& j) const { q[slot] = j; }
};

// First error wins.
__device__ __forceinline__ void set_error(DevStats* st, int code) { atomicCAS(&st->error, 0, code); }

// ---------------------------------------------------------------- streaming warp
template <bool REC>
__device__ __forceinline__ void stream_role(const FusedArgs& a, StreamWarp& W, int lane)
{
    auto grab = [&]() -> int {
        unsigned v = 0;
        if (lane == 0) v = atomicAdd(&a.ctr->item_next, 1u);
        return (int)__shfl_sync(kFull, v, 0);
    };
    auto item_of = [&](int i) -> int4 { return i < a.nitems ? a.items[i] : make_int4(0, 0, 0, -2); };

    // current item (being computed) and next item (taken ahead for the loads)
    int icur = grab();
    int4 cur = item_of(icur);
    int inxt = icur < a.nitems ? grab() : a.nitems;
    int4 nxt = item_of(inxt);
    // loader position: lrel 0 = rows of cur, 1 = rows of nxt, 2 = none known yet
    int lrel = 0, lrow = cur.z - 1;
    unsigned kL = 0, kC = 0;          // loads issued, loads released (load k goes to slot k % kFusedStages)
    unsigned kW = 0xffffffffu;        // load withheld by the test hook
    const long long wait_ns = a.wait_ns;

    // keep up to kFusedStages row loads issued and not yet released
    auto pump = [&]() {
        while (kL - kC < (unsigned)kFusedStages) {
            int4 it;
            int idx;
            if (lrel == 0) { it = cur; idx = icur; }
            else if (lrel == 1) { it = nxt; idx = inxt; }
            else break;
            if (idx >= a.nitems) break;
            const int sl = (int)(kL % kFusedStages);
            const bool skip = a.withhold_load >= 0 && idx == 0 && lrow - (it.z - 1) == a.withhold_load;
            if (skip) kW = kL;
            if (lane == 0 && !skip) {
                mbar_expect_tx(&W.full[sl], kRowBytes);
                tma_load_rows(&a.maps[2 * it.x + a.parity], W.ring[sl], &W.full[sl], it.y * kTmaW - kTmaHalo,
                              lrow + 1);
            }
            ++kL;
            if (++lrow > it.w) {
                ++lrel;
                lrow = lrel == 1 ? nxt.z - 1 : 0;
            }
        }
    };
    auto wait_load = [&](unsigned k) -> bool {
        const bool got = mbar_wait_ns(&W.full[k % kFusedStages], (k / kFusedStages) & 1u, wait_ns);
        return __all_sync(kFull, got);
    };
    // release every load before `k` (their values have been used by every lane)
    auto release_to = [&](unsigned k) {
        __syncwarp();
        kC = k;
        pump();
    };

    WarpQueueSink sink{W.queue, 0};
    // publish the top `count` (1..32) nodes of the warp's queue as one batch
    // (lanes beyond count write empty jobs), queued for block (batch mod blocks)
    auto push_batch = [&](int count) {
        __syncwarp();
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(&a.ctr->batch_tail, 1u);
        b = __shfl_sync(kFull, b, 0);
        if (b >= (unsigned)a.batch_cap) {   // cannot happen (capacity counts every warp's last batch)
            if (lane == 0) set_error(&a.stats[0], 3);
            sink.n -= count;
            return;
        }
        NewtonJob jb;
        if (lane < count) {
            jb = W.queue[sink.n - count + lane];
        } else {
            jb.prob = -1;
            jb.node = 0;
            jb.m0 = jb.theta = 0.0;
        }
        a.jobs[(size_t)b * 32 + lane] = jb;
        sink.n -= count;
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const unsigned tgt = b % gridDim.x;
            const unsigned slot = atomicAdd(a.bq_tail + (size_t)tgt * kBqStride, 1u);
            atomicExch(a.bq + (size_t)tgt * a.bq_cap + slot, b + 1u);
        }
    };

    const float wP[3] = {(float)d2_w(0), (float)d2_w(1), (float)d2_w(5)};
    const int col = kTmaHalo + 4 * lane;   // offset of this lane's first column in a slot's plane row
    bool ok = true;
    DevStats* st_err = nullptr;
    // energy, flux and node counts of the rows this warp computed for one
    // problem, added to the problem's accumulators when the problem changes
    // and at the end (the fixed-point sums make the grouping irrelevant)
    Acc<float> acc;
    TileSums ts;
    DevStats* st_acc = nullptr;
    pump();
    while (ok && icur < a.nitems) {
        const int pi = cur.x, ya = cur.z, yb = cur.w;
        const Problem& pb = a.probs[pi];
        DevStats* st = &a.stats[pb.stats];
        st_err = st;
        if (st != st_acc) {
            if (st_acc) flush_tile_sums<float>(acc, ts, st_acc, lane);
            acc = Acc<float>();
            ts = TileSums();
            st_acc = st;
        }
        const int nx = pb.nx, ny = pb.ny;
        const int segx = cur.y * kTmaW;
        const int x0 = segx + 4 * lane;
        const bool interior_x = segx > 0 && segx + kTmaW < nx;
        const float omc = (float)(1.0 - pb.omega);
        const float om_f = (float)pb.omega;
        const double omc_d = 1.0 - pb.omega;
        const float thr_f = (float)pb.sat;
        float* dst = static_cast<float*>(pb.state[a.parity ^ 1]);
        const long long pl = pb.plane, pitch = pb.pitch;
        // load index of row y of this item: k0 + (y - ya) + 1 (row ya - 1 is load k0)
        const unsigned k0 = kC;

        // row ya - 1: the planes pulled along +y into row ya
        float c2[4], c5[4], c6[4], r4[4], r7[4], r8[4];
        if (!(ok = wait_load(k0))) break;
        {
            const float* s = W.ring[k0 % kFusedStages] + col;
            float t[4];
            ld4(s + 2 * kRowBox, c2);
            ld4(s + 5 * kRowBox, t);
            c5[0] = s[5 * kRowBox - 1]; c5[1] = t[0]; c5[2] = t[1]; c5[3] = t[2];
            ld4(s + 6 * kRowBox, t);
            c6[0] = t[1]; c6[1] = t[2]; c6[2] = t[3]; c6[3] = s[6 * kRowBox + 4];
        }
        // row ya: its planes 4, 7, 8 (unshifted, for theta of row ya)
        if (!(ok = wait_load(k0 + 1))) break;
        {
            const float* s = W.ring[(k0 + 1) % kFusedStages] + col;
            ld4(s + 4 * kRowBox, r4);
            ld4(s + 7 * kRowBox, r7);
            ld4(s + 8 * kRowBox, r8);
        }
        for (int y = ya; y < yb; ++y) {
            const unsigned ky = k0 + 1 + (unsigned)(y - ya);   // load of row y
            if (!(ok = wait_load(ky + 1))) break;
            const float* s0 = W.ring[ky % kFusedStages] + col;         // row y
            const float* s1 = W.ring[(ky + 1) % kFusedStages] + col;   // row y + 1
            float u0[4], u1[4], u2[4], u3[4], u5[4], u6[4], n4[4], n7[4], n8[4];
            ld4(s0 + 0 * kRowBox, u0);
            ld4(s0 + 1 * kRowBox, u1);
            ld4(s0 + 2 * kRowBox, u2);
            ld4(s0 + 3 * kRowBox, u3);
            ld4(s0 + 5 * kRowBox, u5);
            ld4(s0 + 6 * kRowBox, u6);
            const float e1 = s0[1 * kRowBox - 1];   // Omega_1(x0 - 1, y)
            const float e3 = s0[3 * kRowBox + 4];   // Omega_3(x0 + 4, y)
            const float e5 = s0[5 * kRowBox - 1];   // Omega_5(x0 - 1, y), for row y + 1
            const float e6 = s0[6 * kRowBox + 4];   // Omega_6(x0 + 4, y), for row y + 1
            ld4(s1 + 4 * kRowBox, n4);
            ld4(s1 + 7 * kRowBox, n7);
            ld4(s1 + 8 * kRowBox, n8);
            const float e7 = s1[7 * kRowBox + 4];   // Omega_7(x0 + 4, y + 1)
            const float e8 = s1[8 * kRowBox - 1];   // Omega_8(x0 - 1, y + 1)
            // pulled values q_i(x) = Omega_i(x - e_i)
            float qf[9][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                qf[0][k] = u0[k];
                qf[2][k] = c2[k];
                qf[4][k] = n4[k];
                qf[5][k] = c5[k];
                qf[6][k] = c6[k];
            }
            qf[1][0] = e1; qf[1][1] = u1[0]; qf[1][2] = u1[1]; qf[1][3] = u1[2];
            qf[3][0] = u3[1]; qf[3][1] = u3[2]; qf[3][2] = u3[3]; qf[3][3] = e3;
            qf[7][0] = n7[1]; qf[7][1] = n7[2]; qf[7][2] = n7[3]; qf[7][3] = e7;
            qf[8][0] = e8; qf[8][1] = n8[0]; qf[8][2] = n8[1]; qf[8][3] = n8[2];
            const GlobalRowOut<float, 4> out{dst + (long long)(y + 1) * pitch + x0, pl};
            if (pb.method == 1)
                row_update_eebm<float, 4, REC, true>(pb, y, x0, qf, u0, u1, u2, u3, r4, u5, u6, r7, r8, out, a.rec,
                                                     acc, ts, omc, wP, nx, ny);
            else if (interior_x && y > 0 && y < ny - 1)
                row_update<float, 4, REC, false>(pb, y, x0, lane, qf, u0, u1, u2, u3, r4, u5, u6, r7, r8, out, a.rec,
                                                 acc, ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx, ny);
            else
                row_update<float, 4, REC, true>(pb, y, x0, lane, qf, u0, u1, u2, u3, r4, u5, u6, r7, r8, out, a.rec,
                                                acc, ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx, ny);
            // registers for row y + 1
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                c2[k] = u2[k];
                r4[k] = n4[k];
                r7[k] = n7[k];
                r8[k] = n8[k];
            }
            c5[0] = e5; c5[1] = u5[0]; c5[2] = u5[1]; c5[3] = u5[2];
            c6[0] = u6[1]; c6[1] = u6[2]; c6[2] = u6[3]; c6[3] = e6;
            release_to(ky + 1);   // rows up to y (and, in the first row, row ya - 1)
            while (sink.n >= 32) push_batch(32);
        }
        if (!ok) break;
        release_to(k0 + 2 + (unsigned)(yb - ya));   // row yb (its planes 4, 7, 8 were read for row yb - 1)
        // next item
        icur = inxt;
        cur = nxt;
        inxt = icur < a.nitems ? grab() : a.nitems;
        nxt = item_of(inxt);
        if (lrel == 2) {
            lrel = 1;
            lrow = nxt.z - 1;
        } else {
            lrel = 0;
        }
        pump();
    }
    if (!ok) {
        if (lane == 0) set_error(st_err ? st_err : &a.stats[0], 4);   // LBM_ERR_TIMEOUT
        // the row loads still in flight land before the warp may exit
        for (unsigned k = kC; k < kL; ++k)
            if (k != kW) (void)mbar_wait_ns(&W.full[k % kFusedStages], (k / kFusedStages) & 1u, wait_ns);
    }
    if (st_acc) flush_tile_sums<float>(acc, ts, st_acc, lane);
    if (sink.n > 0) push_batch(sink.n);
    // every batch of this warp is queued (and fenced) before it stops streaming
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicSub(&a.ctr->streaming, 1u);
}

// ---------------------------------------------------------------- Newton warp
template <bool REC>
__device__ __forceinline__ void newton_role(const FusedArgs& a, unsigned int* bq_head, int lane)
{
    volatile unsigned int* my_tail = a.bq_tail + (size_t)blockIdx.x * kBqStride;
    unsigned int* my_q = a.bq + (size_t)blockIdx.x * a.bq_cap;
    const long long wait_ns = a.wait_ns;

    // Newton statistics of the batches this warp solved for one problem, kept
    // in registers (the same in every lane) and added to the problem's
    // accumulators when the problem changes and at the end
    int pend_sidx = -1;
    Fx pend_e{0, 0ull};
    unsigned long long pend_n = 0, pend_its = 0;
    int pend_mx = 0;
    auto flush_pending = [&]() {
        if (pend_sidx >= 0 && lane == 0) {
            DevStats* st = &a.stats[pend_sidx];
            StepStripe* c = my_stripe(st);
            acc_add_fx(&c->energy, pend_e);
            atomicAdd(&c->newton, pend_n);
            atomicAdd(&c->iters, pend_its);
            atomicMax(&st->cur_maxit, pend_mx);
        }
        pend_sidx = -1;
        pend_e = Fx{0, 0ull};
        pend_n = pend_its = 0;
        pend_mx = 0;
    };
    auto account = [&](const NewtonResult& r) {
        const unsigned valid = __ballot_sync(kFull, r.sidx >= 0);
        if (!valid) return;
        const int s0 = __shfl_sync(kFull, r.sidx, __ffs(valid) - 1);
        if (!__all_sync(kFull, r.sidx < 0 || r.sidx == s0)) {   // several problems in one batch
            flush_pending();
            newton_group_add(r, a.stats);
            return;
        }
        if (pend_sidx != s0) {
            flush_pending();
            pend_sidx = s0;
        }
        Fx e = r.sidx >= 0 ? r.e : Fx{0, 0ull};
        int its = r.sidx >= 0 ? r.it : 0, mx = its;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Fx v;
            v.hi = __shfl_xor_sync(kFull, e.hi, o);
            v.lo = __shfl_xor_sync(kFull, e.lo, o);
            fx_add(e, v);
            its += __shfl_xor_sync(kFull, its, o);
            mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        }
        fx_add(pend_e, e);
        pend_n += (unsigned long long)__popc(valid);
        pend_its += (unsigned long long)its;
        pend_mx = max(pend_mx, mx);
    };
    // claim one waiting batch of this block's queue, if any, and solve it;
    // true if one was solved
    auto serve = [&]() -> bool {
        int claim = -1;
        if (lane == 0) {
            const unsigned t = *my_tail;
            const unsigned h = *reinterpret_cast<volatile unsigned*>(bq_head);
            if (h < t && atomicCAS(bq_head, h, h + 1) == h) claim = (int)h;
        }
        claim = __shfl_sync(kFull, claim, 0);
        if (claim < 0) return false;
        unsigned e = 0;
        if (lane == 0) {
            volatile unsigned* rf = my_q + claim;
            e = *rf;
            if (e == 0u) {
                const unsigned long long t0 = global_ns();
                while ((e = *rf) == 0u) {
                    if ((long long)(global_ns() - t0) > wait_ns) break;
                    __nanosleep(64);
                }
            }
            *rf = 0u;   // cleared for the next launch
            __threadfence();
        }
        e = __shfl_sync(kFull, e, 0);
        if (e == 0u) {
            if (lane == 0) set_error(&a.stats[0], 4);   // LBM_ERR_TIMEOUT
            return false;
        }
        const long long* jp = reinterpret_cast<const long long*>(a.jobs + (size_t)(e - 1u) * 32 + lane);
        NewtonJob jb;
        long long* jw = reinterpret_cast<long long*>(&jb);
        jw[0] = __ldcg(jp);
        jw[1] = __ldcg(jp + 1);
        jw[2] = __ldcg(jp + 2);
        NewtonResult r;
        if (jb.prob >= 0) r = newton_job_apply<float, REC, 9>(jb, a.probs[jb.prob], a.parity, a.rec, a.stats);
        account(r);
        return true;
    };

    // serve until no warp streams and this block's queue is empty (no batch
    // can be queued after the last streaming warp stops)
    const unsigned long long t0 = global_ns();
    unsigned sleep_ns = 64;
    for (;;) {
        if (serve()) {
            sleep_ns = 64;
            continue;
        }
        int done = 0;
        if (lane == 0) {
            const unsigned str = *reinterpret_cast<volatile unsigned*>(&a.ctr->streaming);
            __threadfence();
            done = (str == 0u && *reinterpret_cast<volatile unsigned*>(bq_head) >= *my_tail) ? 1 : 0;
            if (!done && (long long)(global_ns() - t0) > wait_ns) {
                set_error(&a.stats[0], 4);   // LBM_ERR_TIMEOUT
                done = 1;
            }
        }
        if (__shfl_sync(kFull, done, 0)) break;
        __nanosleep(sleep_ns);
        sleep_ns = min(sleep_ns * 2u, 2048u);
    }
    flush_pending();
}

template <bool REC>
__global__ void __launch_bounds__(kFusedThreads, 1) d2q9_fused_kernel(const FusedArgs a)
{
    extern __shared__ __align__(128) unsigned char fused_smem[];
    __shared__ unsigned int bq_head;   // batches of this block's queue claimed so far
    __shared__ bool last;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) bq_head = 0u;
    if (warp < kStreamWarps && lane == 0) {
        StreamWarp& W = reinterpret_cast<StreamWarp*>(fused_smem)[warp];
        for (int k = 0; k < kFusedStages; ++k) mbar_init(&W.full[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (warp < kStreamWarps)
        stream_role<REC>(a, reinterpret_cast<StreamWarp*>(fused_smem)[warp], lane);
    else
        newton_role<REC>(a, &bq_head, lane);

    // this block's queue is empty and no warp streams: reset its tail.  The
    // last block publishes every problem's step statistics and resets the counters.
    __syncthreads();
    if (threadIdx.x == 0) {
        a.bq_tail[(size_t)blockIdx.x * kBqStride] = 0u;
        __threadfence();
        last = atomicAdd(&a.ctr->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        for (int p = threadIdx.x; p < a.nprob; p += blockDim.x) publish_stats(&a.stats[a.probs[p].stats], &a.probs[p]);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            a.ctr->item_next = 0u;
            a.ctr->streaming = gridDim.x * kStreamWarps;   // the next launch's streaming warps
            a.ctr->batch_tail = 0u;
            a.ctr->ticket = 0u;
        }
    }
}

static bool fused_attr_set(int dev)
{
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) return false;
    if (!done[dev]) {
        if (cudaFuncSetAttribute(d2q9_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(d2q9_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem) !=
                cudaSuccess)
            return false;
        done[dev] = true;
    }
    return true;
}

int d2q9_fused_grid()
{
    int dev = 0, sms = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || !fused_attr_set(dev)) return 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_fused_kernel<false>, kFusedThreads, kFusedSmem);
    return n > 0 ? n * sms : 0;
}

int d2q9_fused_warps() { return kStreamWarps; }

cudaError_t launch_d2q9_fused(const FusedArgs& a, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!fused_attr_set(dev)) return cudaErrorInvalidValue;
    static int grid[64] = {0};
    if (dev >= 64) return cudaErrorInvalidValue;
    if (!grid[dev]) grid[dev] = d2q9_fused_grid();
    if (grid[dev] <= 0) return cudaErrorInvalidConfiguration;
    // cooperative: every block is resident, or the launch fails (warps wait for one another)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid[dev]);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = kFusedSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.rec) return cudaLaunchKernelEx(&cfg, d2q9_fused_kernel<true>, a);
    return cudaLaunchKernelEx(&cfg, d2q9_fused_kernel<false>, a);
}

}  // namespace lbm
