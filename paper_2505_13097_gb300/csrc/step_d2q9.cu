// Fused D2Q9 IREBM step: one kernel launch per time step of Algorithm 3.
//
// The state is the post-collision population Omega_i (Eq. 12), SoA planes.
// For every node y a step does
//   pull       q_i(y) = Omega_i(y - e_i)                       (Algorithm 3, streaming)
//   closures   missing q_i at wall nodes (Sec. 4.2, Eq. 15 and bounce-back)
//   moments    m0 = sum_i q_i, theta(y) = sum_i Omega_i(y)       (sum Omega = M0(f))
//   Newton     theta' = root of Eq. (14) from theta (Algorithm 3)
//   update     f~_i = q_i + w_i (phi(theta) - phi(theta'))/Ste  (Eq. 13)
//   collision  Omega~_i = (1-omega) f~_i + omega w_i theta'     (Eq. 12 of the next step)
// which folds into Omega~_i = (1-omega) q_i + w_i c with c = theta' - (1-omega) m0.
//
// Work unit: a warp tile = one segment of 32*N consecutive x nodes (N = 4
// floats or 2 doubles per thread, one 128-bit load per plane and row) times
// tile_h rows.  The warp marches up its rows keeping the rows it still needs
// in registers: planes with e_y = +1 are pulled from row y-1 (kept from the
// previous row), planes with e_y = -1 from row y+1 (loaded one row ahead and
// kept for the moments of the next row).  Shifts by e_x = +-1 go through warp
// shuffles; lanes 0 and 31 fetch the one element beyond the segment.  Every
// population is read once and written once per step (plus one halo row per
// tile for the six planes with e_y != 0).
//
// FP32 form: populations stored and relaxed in FP32; m0 and theta summed as
// float-float (exact to ~2^-48); the Newton solve in FP64.  Nodes where theta
// and m0 both lie beyond kSat*delta on the same side of the melting point
// take the exact saturated branch (phi = 0 or 1 on both sides of Eq. 14, so
// theta' = m0 and the source vanishes) without any FP64 work.
// FP64 form: everything in FP64 (the saturation test uses the integer pipe).
#include <algorithm>

#include "d2q9_row.cuh"

namespace lbm {

__device__ __forceinline__ void ldg4(const float* p, float (&v)[4])
{
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

// ---------------------------------------------------------------- direct tile
// Same update with rows loaded straight from global memory into registers:
// 2 floats (FP32 form) or 1 double per thread, so a warp covers 256 bytes of
// each plane row and the kernel needs few registers and no shared memory; many
// resident warps keep enough rows in flight.  Planes pulled along +y come from
// the previous row (kept shifted in registers), planes pulled along -y from the
// next row (loaded one row ahead and kept for the moments of the next row).
#ifndef LBM_DIRECT_PREFETCH
#define LBM_DIRECT_PREFETCH 1
#endif

template <typename P> struct Vd;
template <> struct Vd<float> { static constexpr int N = 2; };
template <> struct Vd<double> { static constexpr int N = 1; };

__device__ __forceinline__ void ldg_n(const float* p, float (&v)[2])
{
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ldg_n(const double* p, double (&v)[1]) { v[0] = __ldg(p); }

template <typename P, bool REC>
__device__ __forceinline__ void d2q9_tile_direct(const Problem& pb, const P* __restrict__ src, P* __restrict__ dst,
                                                 double* __restrict__ rec, int seg, int ya, int yb, Acc<P>& acc,
                                                 TileSums& ts, int pi, NewtonJob* jobs, unsigned int* job_count)
{
    GlobalJobSink sink{jobs, job_count};
    constexpr int N = Vd<P>::N;
    const int lane = threadIdx.x & 31;
    const int segx = seg * 32 * N;
    const int x0 = segx + lane * N;
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    const bool has_left = segx > 0;
    const bool has_right = segx + 32 * N < pb.nx;
    const bool seg_interior = has_left && has_right;   // no wall column, every node inside
    const P omc = (P)(1.0 - pb.omega);
    const float om_f = pb.omega_f;
    const double omc_d = 1.0 - pb.omega;
    const int nx = pb.nx, ny = pb.ny;
    const P wP[3] = {lat_wp<P>(9, 0), lat_wp<P>(9, 1), lat_wp<P>(9, 5)};
    const float thr_f = pb.sat_f;
    // the state's shift (FP32 form; 0 in FP64)
    const float sh = sizeof(P) == 4 ? __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(src) + pb.tail_off))
                                    : 0.f;

    auto rp = [&](int i, int r) -> const P* { return src + i * pl + (long long)(r + 1) * pitch + x0; };
    auto hl = [&](int i, int r) -> P {
        return (lane == 0 && has_left) ? __ldg(src + i * pl + (long long)(r + 1) * pitch + segx - 1) : (P)0;
    };
    auto hr = [&](int i, int r) -> P {
        return (lane == 31 && has_right) ? __ldg(src + i * pl + (long long)(r + 1) * pitch + segx + 32 * N) : (P)0;
    };

    P up2[N], up5[N], up6[N], cu4[N], cu7[N], cu8[N];
    {
        P t[N];
        ldg_n(rp(2, ya - 1), up2);
        ldg_n(rp(5, ya - 1), t);
        from_left<P, N>(t, hl(5, ya - 1), lane, up5);
        ldg_n(rp(6, ya - 1), t);
        from_right<P, N>(t, hr(6, ya - 1), lane, up6);
        ldg_n(rp(4, ya), cu4);
        ldg_n(rp(7, ya), cu7);
        ldg_n(rp(8, ya), cu8);
    }
    // loads of one row: planes 0,1,3,2,5,6 at row y, planes 4,7,8 at row y+1, and
    // the elements beyond the segment for the planes shifted along x
    struct RowLoads {
        P r0[N], r1[N], r3[N], c2[N], c5[N], c6[N], n4[N], n7[N], n8[N];
        P h1, h3, h5, h6, h7, h8;
    };
    auto issue = [&](RowLoads& L, int y) {
        ldg_n(rp(0, y), L.r0);
        ldg_n(rp(1, y), L.r1);
        ldg_n(rp(3, y), L.r3);
        ldg_n(rp(2, y), L.c2);
        ldg_n(rp(5, y), L.c5);
        ldg_n(rp(6, y), L.c6);
        ldg_n(rp(4, y + 1), L.n4);
        ldg_n(rp(7, y + 1), L.n7);
        ldg_n(rp(8, y + 1), L.n8);
        L.h1 = hl(1, y);
        L.h3 = hr(3, y);
        L.h5 = hl(5, y);
        L.h6 = hr(6, y);
        L.h7 = hr(7, y + 1);
        L.h8 = hl(8, y + 1);
    };
    RowLoads cur;
    issue(cur, ya);
    for (int y = ya; y < yb; ++y) {
        // next row's loads first, so they are in flight during this row's arithmetic
        RowLoads nxt;
        if (LBM_DIRECT_PREFETCH && y + 1 < yb) issue(nxt, y + 1);
        P qf[9][N];
        {
            P s[N];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                qf[0][k] = cur.r0[k]; qf[2][k] = up2[k]; qf[4][k] = cur.n4[k]; qf[5][k] = up5[k]; qf[6][k] = up6[k];
            }
            from_left<P, N>(cur.r1, cur.h1, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[1][k] = s[k];
            from_right<P, N>(cur.r3, cur.h3, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[3][k] = s[k];
            from_right<P, N>(cur.n7, cur.h7, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[7][k] = s[k];
            from_left<P, N>(cur.n8, cur.h8, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[8][k] = s[k];
        }
        if (pb.method == 1)
            row_update_eebm<P, N, REC, true>(pb, y, x0, qf, cur.r0, cur.r1, cur.c2, cur.r3, cu4, cur.c5, cur.c6, cu7,
                                             cu8, GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec,
                                             acc, ts, omc, wP, nx, ny, sh);
        else if (seg_interior && y > 0 && y < ny - 1)
            row_update<P, N, REC, false>(pb, y, x0, lane, qf, cur.r0, cur.r1, cur.c2, cur.r3, cu4, cur.c5, cur.c6, cu7,
                                         cu8, GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec, acc,
                                         ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx, ny, sh);
        else
            row_update<P, N, REC, true>(pb, y, x0, lane, qf, cur.r0, cur.r1, cur.c2, cur.r3, cu4, cur.c5, cur.c6, cu7,
                                        cu8, GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec, acc,
                                        ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx, ny, sh);
        // roll the register window
#pragma unroll
        for (int k = 0; k < N; ++k) { up2[k] = cur.c2[k]; cu4[k] = cur.n4[k]; cu7[k] = cur.n7[k]; cu8[k] = cur.n8[k]; }
        from_left<P, N>(cur.c5, cur.h5, lane, up5);
        from_right<P, N>(cur.c6, cur.h6, lane, up6);
        if (LBM_DIRECT_PREFETCH) {
            cur = nxt;
        } else if (y + 1 < yb) {
            issue(cur, y + 1);
        }
    }
}

template <typename P, bool REC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4) d2q9_step_kernel(StepArgs a)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int slot = warp; slot < a.nslots; slot += nwarps) {
        int pi, t;
        if (a.schedule) {
            const int2 s = a.schedule[slot];
            pi = s.x;
            t = s.y;
        } else {
            pi = 0;
            t = slot;
        }
        const Problem& pb = a.probs[pi];
        DevStats* st = &a.stats[pb.stats];
        const int seg = t % pb.nseg;
        const int strip = t / pb.nseg;
        const int ya = strip * pb.tile_h;
        const int yb = min(pb.ny, ya + pb.tile_h);
        const P* src = static_cast<const P*>(pb.state[a.parity]);
        P* dst = static_cast<P*>(pb.state[a.parity ^ 1]);
        Acc<P> acc;
        TileSums ts;
        d2q9_tile_direct<P, REC>(pb, src, dst, a.rec, seg, ya, yb, acc, ts, pi, a.jobs, a.job_count);
        flush_tile_sums<P>(acc, ts, st, lane);
    }
    // statistics are published by the job kernel that follows every step
}

// ---------------------------------------------------------------- flat step
// Single-problem FP32 step.  A tile is 128 columns x 8 rows; a block (8
// warps) computes one tile, one row per warp, four consecutive columns per
// lane; consecutive blocks take the strips of one row band before the next
// band.  Every pull
// is a read-only load from global memory: for row y a lane loads the nine
// planes of row y (its four columns; one 128-bit load each), planes 2, 5, 6
// of row y - 1 and 4, 7, 8 of row y + 1, and the six elements just left or
// right of its columns that the diagonal and horizontal pulls need.  The
// rows above and below are also loaded by the neighbouring warps and tiles at
// about the same time, so L1 and L2 serve them and DRAM sees each population
// read once.  No shared memory, no barrier inside the loop: many independent
// 128-bit loads per thread keep the memory system busy.  Loads left of column
// 0 or right of the last column read other rows' elements; they only feed
// directions that the wall closures replace.  The energy and node-count sums
// of a block are combined once per launch.
// The loads of one row of the flat step: the nine planes of row y (u), and
// the pulled values q_i(x) = Omega_i(x - e_i) (qf), for four columns x0..x0+3.
__device__ __forceinline__ void flat_load_row(const float* __restrict__ row, long long pitch, long long pl,
                                              float (&u)[9][4], float (&qf)[9][4])
{
    const float* up = row - pitch;   // row y - 1
    const float* dn = row + pitch;   // row y + 1
#pragma unroll
    for (int i = 0; i < 9; ++i) ldg4(row + i * pl, u[i]);
    float a2[4], a5[4], a6[4], b4[4], b7[4], b8[4];
    ldg4(up + 2 * pl, a2);
    ldg4(up + 5 * pl, a5);
    ldg4(up + 6 * pl, a6);
    ldg4(dn + 4 * pl, b4);
    ldg4(dn + 7 * pl, b7);
    ldg4(dn + 8 * pl, b8);
    const float e1 = __ldg(row + 1 * pl - 1);   // Omega_1(x0 - 1, y)
    const float e3 = __ldg(row + 3 * pl + 4);   // Omega_3(x0 + 4, y)
    const float e5 = __ldg(up + 5 * pl - 1);    // Omega_5(x0 - 1, y - 1)
    const float e6 = __ldg(up + 6 * pl + 4);    // Omega_6(x0 + 4, y - 1)
    const float e7 = __ldg(dn + 7 * pl + 4);    // Omega_7(x0 + 4, y + 1)
    const float e8 = __ldg(dn + 8 * pl - 1);    // Omega_8(x0 - 1, y + 1)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        qf[0][k] = u[0][k];
        qf[2][k] = a2[k];
        qf[4][k] = b4[k];
    }
    qf[1][0] = e1; qf[1][1] = u[1][0]; qf[1][2] = u[1][1]; qf[1][3] = u[1][2];
    qf[3][0] = u[3][1]; qf[3][1] = u[3][2]; qf[3][2] = u[3][3]; qf[3][3] = e3;
    qf[5][0] = e5; qf[5][1] = a5[0]; qf[5][2] = a5[1]; qf[5][3] = a5[2];
    qf[6][0] = a6[1]; qf[6][1] = a6[2]; qf[6][2] = a6[3]; qf[6][3] = e6;
    qf[7][0] = b7[1]; qf[7][1] = b7[2]; qf[7][2] = b7[3]; qf[7][3] = e7;
    qf[8][0] = e8; qf[8][1] = b8[0]; qf[8][2] = b8[1]; qf[8][3] = b8[2];
}

// What the scalar path adds for one node to its lane's sums.
struct ColdSums {
    ff e{0.f, 0.f};      // energy term (saturated and EEBM nodes: less the state's shift)
    ff flux{0.f, 0.f};   // boundary flux
    int liquid = 0, shifted = 0, dir = -1;
};

// One node (x, y), 1 <= y <= ny-2, of the flat step that the vector path
// leaves out: a node on the W or E wall, or any node of a four-column group
// that holds one (or reaches past nx).  The arithmetic of row_update /
// row_update_eebm for one FP32 node, with scalar loads and stores; a Newton
// node takes a job slot of its own.  Run by the wall kernel, one node per
// thread, so that the flat kernel carries no closure code.
__device__ __forceinline__ void flat_cold_node(const Problem& pb, int pi, const float* __restrict__ src,
                                                   float* __restrict__ dst, double* __restrict__ rec, int x, int y,
                                                   float sh, NewtonJob* jobs, unsigned int* job_count, ColdSums& cs)
{
    const long long pl = pb.plane, pitch = pb.pitch;
    const long long at = (long long)(y + 1) * pitch + x;
    float u[9], q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        u[i] = __ldg(src + i * pl + at);
        q[i] = __ldg(src + i * pl + at - d2_ey(i) * pitch - d2_ex(i));   // Omega_i(x - e_i)
    }
    int wall = -1;
    if (x == 0 || x == pb.nx - 1) cs.flux = wall_closure_f(q, u, x, y, pb, wall, sh);
    const float omc = pb.omc_f;
    const float wP[3] = {d2_wf(0), d2_wf(1), d2_wf(5)};
    float* d = dst + at;
    if (pb.method == 1) {
        // EEBM (row_update_eebm)
        float Hs = 0.f;
#pragma unroll
        for (int i = 8; i >= 0; --i) Hs += q[i];
        const float om = 1.0f - omc;
        const float H = Hs + sh;
        const float th = eebm_theta(H, (float)pb.inv_ste);
        d[0] = fmaf(omc, q[0], om * (H - (1.0f - wP[0]) * th - wP[0] * sh));
        const float tr = th - sh;
#pragma unroll
        for (int i = 1; i < 9; ++i) d[i * pl] = fmaf(omc, q[i], om * (i <= 4 ? wP[1] : wP[2]) * tr);
        cs.e = ff{Hs, 0.f};
        cs.shifted = 1;
        if (rec) rec[(long long)y * pitch + x] = (double)th;
        return;
    }
    const float tf = approx_sum<float>(u) + sh;
    float mf = 0.f;
#pragma unroll
    for (int i = 8; i >= 0; --i) mf += q[i];
    const float mt = mf + sh;
    const float thr_f = pb.sat_f;
    const float marg = 1e-5f * (1.0f + fabsf(tf));
    const bool sat_liq = tf >= thr_f + marg && mt >= thr_f + marg;
    const bool sat_sol = tf <= -thr_f - marg && mt <= -thr_f - marg;
    float c;
    double thn;
    if (wall >= 0) {
        // Dirichlet node: theta' = theta_D; c less omega sh
        ff mm{0.f, 0.f};
#pragma unroll
        for (int i = 8; i >= 0; --i) ff_add(mm, q[i]);
        c = ((pb.wall_th_hi[wall] - sh) - omc * mm.hi) + (pb.wall_th_lo[wall] - omc * mm.lo);
        cs.e = ff{pb.wall_th_hi[wall], pb.wall_th_lo[wall]};
        cs.dir = wall;
        thn = pb.wall_theta[wall];
    } else if (sat_liq || sat_sol) {
        c = pb.omega_f * mf;
        cs.e = ff{mf, 0.f};
        cs.shifted = 1;
        cs.liquid = sat_liq ? 1 : 0;
        thn = (double)mf + (double)sh;
    } else {
        // the local Newton solve of Eq. (14) is deferred: q stored unrelaxed
        NewtonJob jb;
        jb.prob = pi;
        jb.node = y * pb.nx + x;
        jb.m0 = jb.theta = 0.0;
        jobs[atomicAdd(job_count, 1u)] = jb;
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i * pl] = q[i];
        if (rec) rec[(long long)y * pitch + x] = 0.0;
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i * pl] = fmaf(omc, q[i], wP[i == 0 ? 0 : (i <= 4 ? 1 : 2)] * c);
    if (rec) rec[(long long)y * pitch + x] = thn;
}

#ifndef LBM_FLAT_MINB
#define LBM_FLAT_MINB 3   // resident blocks per SM the register budget is fitted to
#endif
// Rows 1 .. ny-2 of every 128-column strip; IREBM (Algorithm 3) or, with
// EEBM, Algorithm 2.  A block takes one tile of 128 columns x 8 rows (single
// problem: tile t = strip t % nsegs, rows 8 (t / nsegs) + warp; batches: the
// tile table a.ftiles, entry (problem, strip, first row)).  Lanes whose four
// columns are all inside (1 <= x <= nx-2) run the vector path below; a lane
// whose group holds column 0 or nx-1 or reaches past nx leaves it and runs
// flat_cold_node for each of its nodes inside the lattice.  Rows 0 and ny-1
// are the wall-row kernel's.
template <bool REC, bool EEBM>
__global__ void __launch_bounds__(256, LBM_FLAT_MINB) d2q9_flat_kernel(const StepArgs a)
{
    __shared__ WarpSums wsum[8];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    int pi, seg, y;
    if (a.ftiles) {
        const int4 t = a.ftiles[blockIdx.x];
        pi = t.x;
        seg = t.y;
        y = t.z + warp;
    } else {
        const int nsegs = a.nsegc > 0 ? a.nsegc : a.probs[0].pitch / 128;
        pi = 0;
        seg = a.seg0 + blockIdx.x % nsegs;
        y = (blockIdx.x / nsegs) * 8 + warp;
    }
    const Problem& pb = a.probs[pi];
    const int nx = pb.nx, ny = pb.ny;
    Acc<float> acc;
    TileSums ts;
    const int x0 = seg * 128 + 4 * lane;
    if (y >= 1 && y < ny - 1) {   // the same for the whole warp
        const long long pl = pb.plane, pitch = pb.pitch;
        const float* __restrict__ src = static_cast<const float*>(pb.state[a.parity]);
        float* __restrict__ dst = static_cast<float*>(pb.state[a.parity ^ 1]);
        const float omc = pb.omc_f;
        const float wP[3] = {d2_wf(0), d2_wf(1), d2_wf(5)};
        const float sh = state_shift(pb, a.parity);   // stored values are Omega_i - w_i sh
        const float* row = src + (y + 1) * pitch + x0;
        float* orow = dst + (y + 1) * pitch + x0;
        // cold: the group holds column 0 or nx-1, or lies (partly) past nx
        const bool cold = x0 == 0 || x0 + 3 >= nx - 1;
        // every load of the vector path stays inside the buffer, cold lanes included
        float u[9][4], qf[9][4];
        flat_load_row(row, pitch, pl, u, qf);
        if constexpr (EEBM) {
            const float om = 1.0f - omc;
            const float inv_ste = (float)pb.inv_ste;
            float hs = 0.f;
            double thn[REC ? 4 : 1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float Hs = 0.f;   // H less the shift
#pragma unroll
                for (int i = 8; i >= 0; --i) Hs += qf[i][k];
                hs += Hs;
                const float H = Hs + sh;
                const float th = eebm_theta(H, inv_ste);
                if constexpr (REC) thn[k] = (double)th;
                qf[0][k] = fmaf(omc, qf[0][k], om * (H - (1.0f - wP[0]) * th - wP[0] * sh));
                const float tr = th - sh;
#pragma unroll
                for (int i = 1; i < 9; ++i) qf[i][k] = fmaf(omc, qf[i][k], om * (i <= 4 ? wP[1] : wP[2]) * tr);
            }
            if (!cold) {
                acc.add_ff(ff{hs, 0.f});
                ts.shifted += 4;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    float o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) o[k] = qf[i][k];
                    stv_n(orow + i * pl, o);
                }
                if constexpr (REC) st_rec<4>(a.rec + (long long)y * pitch + x0, thn);
            }
        } else {
            // interior IREBM nodes: the arithmetic of row_update's interior branch
            const float om_f = pb.omega_f;
            const float thr_f = pb.sat_f;
            float c[4], esum = 0.f;   // the lane's energy terms, less the shift
            bool newton[4];
            bool any_newton = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float uk[9] = {u[0][k], u[1][k], u[2][k], u[3][k], u[4][k], u[5][k], u[6][k], u[7][k], u[8][k]};
                const float tf = approx_sum<float>(uk) + sh;   // theta
                float mf = 0.f;                                  // M0(q) - sh
#pragma unroll
                for (int i = 8; i >= 0; --i) mf += qf[i][k];
                const float mt = mf + sh;
                const float marg = 1e-5f * (1.0f + fabsf(tf));
                const bool sat_liq = tf >= thr_f + marg && mt >= thr_f + marg;
                const bool sat_sol = tf <= -thr_f - marg && mt <= -thr_f - marg;
                newton[k] = !cold && !(sat_liq || sat_sol);
                any_newton |= newton[k];
                c[k] = newton[k] ? 0.f : om_f * mf;   // c - omega sh = omega (m0 - sh)
                if (!newton[k] && !cold) {
                    esum += mf;
                    ts.liquid += sat_liq ? 1 : 0;
                    ts.shifted += 1;
                }
            }
            acc.add_f(esum);   // one float-float addition per lane and row
            float wc[3][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                wc[0][k] = wP[0] * c[k];
                wc[1][k] = wP[1] * c[k];
                wc[2][k] = wP[2] * c[k];
            }
            if (__any_sync(kFull, any_newton)) {
                // nodes that need the local Newton solve: stored unrelaxed, their
                // index appended to the job list (the job kernel forms m0, theta)
                int cnt = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) cnt += newton[k] ? 1 : 0;
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += v;
                }
                GlobalJobSink sink{a.jobs, a.job_count};
                const unsigned base = sink.reserve((unsigned)__shfl_sync(kFull, incl, 31), lane);
                unsigned slot = base + (unsigned)(incl - cnt);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (newton[k]) {
                        NewtonJob jb;
                        jb.prob = pi;
                        jb.node = y * nx + x0 + k;
                        jb.m0 = jb.theta = 0.0;
                        a.jobs[slot++] = jb;
                    }
            }
            if (!cold) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int cl = i == 0 ? 0 : (i <= 4 ? 1 : 2);
                    float o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) o[k] = newton[k] ? qf[i][k] : fmaf(omc, qf[i][k], wc[cl][k]);
                    stv_n(orow + i * pl, o);
                }
                if constexpr (REC) {
                    double thn[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float mf = 0.f;
#pragma unroll
                        for (int i = 8; i >= 0; --i) mf += qf[i][k];
                        thn[k] = newton[k] ? 0.0 : (double)mf + (double)sh;
                    }
                    st_rec<4>(a.rec + (long long)y * pitch + x0, thn);
                }
            }
        }
        // cold lanes: their nodes are the wall kernel's
    }
    const WarpSums w = warp_tile_sums<float>(acc, ts);
    if (lane == 0) wsum[warp] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        WarpSums tot = wsum[0];
        for (int k = 1; k < 8; ++k) add_sums(tot, wsum[k]);
        emit_sums(tot, &a.stats[pb.stats]);
    }
}

// The nodes the flat kernel leaves out, FP32, in two kernels.
//  * d2q9_wall_kernel: rows 0 and ny-1 (the S and N walls) of every
//    128-column strip, one row per warp, the full row update (closures of
//    Sec. 4.2, Newton hand-off, EEBM).  Row r: single problem, strip r / 2,
//    row 0 or ny-1 by r % 2; batches: the table a.wrows, entry (problem,
//    2 strip + (0: row 0, 1: row ny-1)).  Each warp adds its sums to its
//    problem after each row.
//  * d2q9_wall_cols_kernel: in rows 1 .. ny-2, the nodes of the four-column
//    groups that hold column 0 or nx-1 or reach past nx, one node per thread
//    (flat_cold_node): 32 rows per block, eight slots per row (x = 0 .. 3 and
//    x = xe .. xe + 3, xe the group of column nx-1 when it is not the first).
//    Single problem: block b takes rows 1 + 32 b ...; batches: the table
//    a.crows, entry (problem, first row).
template <bool REC>
__global__ void __launch_bounds__(256) d2q9_wall_kernel(const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nrows = a.wrows ? a.nwrows : 2 * (a.probs[0].pitch / 128);
    for (int r = blockIdx.x * 8 + warp; r < nrows; r += gridDim.x * 8) {
        int pi = 0, code = r;
        if (a.wrows) {
            const int2 e = a.wrows[r];
            pi = e.x;
            code = e.y;
        }
        const Problem& pb = a.probs[pi];
        const int nx = pb.nx, ny = pb.ny;
        const long long pl = pb.plane, pitch = pb.pitch;
        const int seg = code >> 1;
        const int y = (code & 1) ? ny - 1 : 0;
        const float* __restrict__ src = static_cast<const float*>(pb.state[a.parity]);
        float* __restrict__ dst = static_cast<float*>(pb.state[a.parity ^ 1]);
        const float omc = pb.omc_f;
        const float om_f = pb.omega_f;
        const double omc_d = 1.0 - pb.omega;
        const float wP[3] = {d2_wf(0), d2_wf(1), d2_wf(5)};
        const float thr_f = pb.sat_f;
        const float sh = state_shift(pb, a.parity);   // stored values are Omega_i - w_i sh
        Acc<float> acc;
        TileSums ts;
        GlobalJobSink sink{a.jobs, a.job_count};
        const int x0 = seg * 128 + 4 * lane;
        float u[9][4], qf[9][4];
        flat_load_row(src + (y + 1) * pitch + x0, pitch, pl, u, qf);
        const GlobalRowOut<float, 4> out{dst + (y + 1) * pitch + x0, pl};
        if (pb.method == 1)
            row_update_eebm<float, 4, REC, true>(pb, y, x0, qf, u[0], u[1], u[2], u[3], u[4], u[5], u[6], u[7],
                                                 u[8], out, a.rec, acc, ts, omc, wP, nx, ny, sh);
        else
            row_update<float, 4, REC, true>(pb, y, x0, lane, qf, u[0], u[1], u[2], u[3], u[4], u[5], u[6], u[7],
                                            u[8], out, a.rec, acc, ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx,
                                            ny, sh);
        flush_tile_sums<float>(acc, ts, &a.stats[pb.stats], lane);
    }
}

// (one node per thread needs far fewer registers than the row update, so more
// blocks fit on an SM than in the rows kernel)
template <bool REC>
__global__ void __launch_bounds__(256) d2q9_wall_cols_kernel(const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    int pi = 0, y0 = 1 + 32 * b;
    if (a.crows) {
        const int2 e = a.crows[b];
        pi = e.x;
        y0 = e.y;
    }
    const Problem& pb = a.probs[pi];
    const int nx = pb.nx, ny = pb.ny;
    const int y = y0 + (threadIdx.x >> 3);
    const int slot = threadIdx.x & 7;
    const int xe = max(4, ((nx - 1) >> 2) << 2);
    const int x = slot < 4 ? slot : xe + slot - 4;
    Acc<float> acc;
    TileSums ts;
    if (y >= 1 && y < ny - 1 && x < nx && (slot >= 4 || x < 4)) {
        ColdSums cs;
        flat_cold_node(pb, pi, static_cast<const float*>(pb.state[a.parity]), static_cast<float*>(pb.state[a.parity ^ 1]),
                       a.rec, x, y, state_shift(pb, a.parity), a.jobs, a.job_count, cs);
        acc.add_ff(cs.e);
        ff_add(ts.flux_f, cs.flux.hi);
        ts.flux_f.lo += cs.flux.lo;
        ts.liquid += cs.liquid;
        ts.shifted += cs.shifted;
        if (cs.dir >= 0) ts.dir_count[cs.dir] += 1;
    }
    flush_tile_sums<float>(acc, ts, &a.stats[pb.stats], lane);
}

// ---------------------------------------------------------------- TMA row pipeline
// Single-problem FP32 step, warp-specialized.  A block owns a strip of
// kTmaW = 128 columns and a contiguous range of rows [ya, yb).  A producer
// warp streams rows of all nine planes into a ring of shared-memory slots
// with TMA tensor loads (136 columns: four more on each side for the pulls
// along x; outside the tensor the hardware fills zeros); a load completes on
// the slot's `full` mbarrier.  Four consumer warps (32 columns each, one node
// per lane) take the pulled values of row y from the slots of rows y-1, y and
// y+1 (shared-memory loads at +-1 column, no shuffles), run the row update
// above, store their outputs straight to global memory, and release the slot
// of row y-1 on its `empty` mbarrier, which the producer waits on before it
// reuses the slot.  The consumers are not synchronized with one another, and
// the ring keeps up to kTmaStages rows in flight per block without holding
// registers.  Every mbarrier wait is bounded: on a timeout the kernel records
// LBM_ERR_TIMEOUT, stops, and the producer waits (bounded) for its own copies
// in flight before it exits.
#ifndef LBM_TMA_STAGES
#define LBM_TMA_STAGES 8
#endif
constexpr int kTmaStages = LBM_TMA_STAGES;
constexpr int kTmaBox = kTmaW + 2 * kTmaHalo;                  // 136 loaded columns
constexpr int kTmaSlot = (9 * kTmaBox * 4 + 127) / 128 * 32;   // floats per slot (128-byte multiple)
constexpr int kTmaConsumers = kTmaW / 32;                       // consumer warps
constexpr int kTmaThreads = kTmaW + 32;                         // + the producer warp
constexpr unsigned kTmaRowBytes = 9u * kTmaBox * 4u;             // bytes one row load delivers

#ifndef LBM_TMA_MIN_BLOCKS
#define LBM_TMA_MIN_BLOCKS 5   // resident blocks per SM the register budget is fitted to
#endif

template <bool REC>
__global__ void __launch_bounds__(kTmaThreads, LBM_TMA_MIN_BLOCKS) d2q9_tma_kernel(const StepArgs a, const __grid_constant__ TmaMaps m)
{
    __shared__ __align__(128) float ring[kTmaStages * kTmaSlot];
    __shared__ __align__(8) unsigned long long full[kTmaStages];
    __shared__ __align__(8) unsigned long long empty[kTmaStages];

    const int pi = 0;
    const int seg = blockIdx.x % m.nsegs;
    const int part = blockIdx.x / m.nsegs;
    const int nyp = a.probs[0].ny;
    const int ya = (int)((long long)nyp * part / m.nparts);
    const int yb = (int)((long long)nyp * (part + 1) / m.nparts);
    const CUtensorMap* lmap = &m.load[a.parity];
    const Problem& pb = a.probs[pi];
    DevStats* st = &a.stats[pb.stats];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int nx = pb.nx, ny = pb.ny;
    const int segx = seg * kTmaW;

    if (tid == 0) {
        for (int k = 0; k < kTmaStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kTmaConsumers);
        }
        fence_mbar_init();
    }
    __syncthreads();
    // row r (ya-1 <= r <= yb) is the k-th load, k = r - ya + 1: slot k % S, use k / S

    if (warp == kTmaConsumers) {
        // ---- producer
        if (lane == 0) {
            int last = -1;   // last k issued
            bool ok = true;
            for (int r = ya - 1; r <= yb; ++r) {
                const int k = r - (ya - 1);
                const int sl = k % kTmaStages;
                if (k >= kTmaStages && !mbar_wait_bounded(&empty[sl], (unsigned)((k / kTmaStages - 1) & 1), m.wait_ns)) {
                    ok = false;
                    break;
                }
                last = k;
                if (k == m.withhold_load && blockIdx.x == 0) continue;   // test hook: this row never arrives
                mbar_expect_tx(&full[sl], kTmaRowBytes);
                tma_load_rows(lmap, ring + sl * kTmaSlot, &full[sl], segx - kTmaHalo, r + 1);
            }
            if (!ok) {
                atomicExch(&st->error, 4);   // LBM_ERR_TIMEOUT
                // the copies still in flight land before the block may exit
                for (int k = max(0, last - kTmaStages + 1); k <= last; ++k)
                    (void)mbar_wait_bounded(&full[k % kTmaStages], (unsigned)((k / kTmaStages) & 1), m.wait_ns);
            }
        }
        return;
    }

    // ---- consumers
    const int x = segx + tid;
    const float omc = pb.omc_f;
    const float om_f = pb.omega_f;
    const double omc_d = 1.0 - pb.omega;
    const float wP[3] = {d2_wf(0), d2_wf(1), d2_wf(5)};
    const float thr_f = pb.sat_f;
    const float sh = state_shift(pb, a.parity);   // stored values are Omega_i - w_i sh
    const int wx0 = segx + warp * 32;   // first column of this warp
    const bool warp_interior_x = wx0 > 0 && wx0 + 31 < nx - 1;
    float* dst = static_cast<float*>(pb.state[a.parity ^ 1]);
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    Acc<float> acc;
    TileSums ts;
    GlobalJobSink sink{a.jobs, a.job_count};
    auto wait_row = [&](int r) -> bool {
        const int k = r - (ya - 1);
        return mbar_wait_bounded(&full[k % kTmaStages], (unsigned)((k / kTmaStages) & 1), m.wait_ns);
    };
    bool ok = wait_row(ya - 1) && wait_row(ya);
    for (int y = ya; ok && y < yb; ++y) {
        ok = wait_row(y + 1);
        if (!ok) break;
        const int km = y - 1 - (ya - 1);
        const float* sm1 = ring + (km % kTmaStages) * kTmaSlot + kTmaHalo + tid;
        const float* s0 = ring + ((km + 1) % kTmaStages) * kTmaSlot + kTmaHalo + tid;
        const float* sp1 = ring + ((km + 2) % kTmaStages) * kTmaSlot + kTmaHalo + tid;
        float u0[1], u1[1], u2[1], u3[1], u4[1], u5[1], u6[1], u7[1], u8[1];
        u0[0] = s0[0 * kTmaBox]; u1[0] = s0[1 * kTmaBox]; u2[0] = s0[2 * kTmaBox];
        u3[0] = s0[3 * kTmaBox]; u4[0] = s0[4 * kTmaBox]; u5[0] = s0[5 * kTmaBox];
        u6[0] = s0[6 * kTmaBox]; u7[0] = s0[7 * kTmaBox]; u8[0] = s0[8 * kTmaBox];
        float qf[9][1];
        qf[0][0] = u0[0];
        qf[1][0] = s0[1 * kTmaBox - 1];    // Omega_1(x - 1, y)
        qf[3][0] = s0[3 * kTmaBox + 1];    // Omega_3(x + 1, y)
        qf[2][0] = sm1[2 * kTmaBox];       // Omega_2(x, y - 1)
        qf[5][0] = sm1[5 * kTmaBox - 1];   // Omega_5(x - 1, y - 1)
        qf[6][0] = sm1[6 * kTmaBox + 1];   // Omega_6(x + 1, y - 1)
        qf[4][0] = sp1[4 * kTmaBox];       // Omega_4(x, y + 1)
        qf[7][0] = sp1[7 * kTmaBox + 1];   // Omega_7(x + 1, y + 1)
        qf[8][0] = sp1[8 * kTmaBox - 1];   // Omega_8(x - 1, y + 1)
        // every lane has read the slot of row y - 1: release it to the producer
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[km % kTmaStages]);
        const GlobalRowOut<float, 1> out{dst + (long long)(y + 1) * pitch + x, pl};
        if (pb.method == 1)
            row_update_eebm<float, 1, REC, true>(pb, y, x, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8, out, a.rec, acc, ts,
                                                 omc, wP, nx, ny, sh);
        else if (warp_interior_x && y > 0 && y < ny - 1)
            row_update<float, 1, REC, false>(pb, y, x, lane, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8, out, a.rec, acc,
                                             ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx, ny, sh);
        else
            row_update<float, 1, REC, true>(pb, y, x, lane, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8, out, a.rec, acc,
                                            ts, pi, sink, omc, om_f, omc_d, wP, thr_f, nx, ny, sh);
    }
    if (!ok && lane == 0) atomicExch(&st->error, 4);   // LBM_ERR_TIMEOUT
    flush_tile_sums<float>(acc, ts, st, lane);
}

// ---------------------------------------------------------------- Newton jobs
// Local Newton solves deferred by the step kernel (Eq. 14, mixed-precision
// form: FP32 then FP64 steps, newton_mixed), one job per lane, consecutive jobs
// per warp; Q = 9 (D2Q9) or 5 (D2Q5) planes.  For each job:
//   theta' = m0 + (phi(theta) - phi(root))/Ste,  c = theta' - (1-omega) m0,
//   Omega~_i = (1-omega) q_i + w_i c   (q_i was stored by the step kernel).
// Energy contributions theta' + phi(theta')/Ste are summed per problem as
// exact 128-bit fixed-point integers (independent of the job order).  The last
// warp to finish publishes the step statistics and clears the job list.
// Threads per block of the job kernel.  Its last block is found with one
// atomic ticket per block, and same-address atomics serialize in L2: with 1,216
// blocks an empty job list still took 16 us, so the grid is kept small (one or
// two blocks of 256 threads per SM; each warp takes jobs grid-stride or from a
// shared cursor).  A solve is a chain of dependent FP64 operations: it needs
// many warps per SM to keep the FP64 pipe busy.  Beside the flat kernel, 64-
// thread blocks at 64 registers (which fit beside its three blocks per SM)
// solved the front band of the 4096^2 melting workload at a third of the rate
// of one 256-thread block per SM, and the step took 14 % longer.  The FP32
// form's kernel is held to 80 registers (three blocks per SM), so that its
// block beside the flat kernel takes the place of one flat block, not two.
#ifndef LBM_JOB_SIDE_WARPS
#define LBM_JOB_SIDE_WARPS 8   // warps per block of the job launch beside the flat kernel
#endif
constexpr int kJobThreads = 256;
constexpr int kJobSideThreads = 32 * LBM_JOB_SIDE_WARPS;
constexpr int kJobMinBlocksF = LBM_JOB_SIDE_WARPS == 2 ? 4 : 3;

// One warp's 32 jobs from `base` of a list of `count` (lanes past the end idle).
template <typename P, bool REC, int Q>
__device__ __forceinline__ void newton_job_group(const JobArgs& a, const NewtonJob* jobs, unsigned base,
                                                 unsigned count, int lane)
{
    const unsigned j = base + lane;
    NewtonResult r;
    if (j < count) {
        const NewtonJob jb = jobs[j];
        r = newton_job_apply<P, REC, Q>(jb, a.probs[jb.prob], a.parity, a.rec, a.stats);
    }
    newton_group_add(r, a.stats);
}

template <typename P, bool REC, int Q>
__global__ void __launch_bounds__(kJobThreads, sizeof(P) == 4 ? kJobMinBlocksF : 1) newton_jobs_kernel(JobArgs a)
{
    // the counts (and the cursor) as independent loads, one round trip
    const unsigned count = *reinterpret_cast<volatile unsigned*>(a.job_count);
    const unsigned count2 = a.jobs2 ? *reinterpret_cast<volatile unsigned*>(a.job_count2) : 0u;
    unsigned cur0 = a.cursor ? *reinterpret_cast<volatile unsigned*>(a.cursor) : 0u;
    const int lane = threadIdx.x & 31;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    if (a.cursor) {
        // shared list: 32 jobs per take; a plain read first, so that a warp
        // that finds the list taken issues no atomic
        volatile unsigned* cur = a.cursor;
        for (bool first = true;; first = false) {
            unsigned base = 0;
            if (lane == 0) {
                base = first ? cur0 : *cur;
                if (base < count) base = atomicAdd(a.cursor, 32u);
            }
            base = __shfl_sync(kFull, base, 0);
            if (base >= count) break;
            newton_job_group<P, REC, Q>(a, a.jobs, base, count, lane);
        }
    } else {
        for (unsigned base = gw * 32; base < count; base += nw * 32)
            newton_job_group<P, REC, Q>(a, a.jobs, base, count, lane);
    }
    if (a.jobs2) {
        for (unsigned base = gw * 32; base < count2; base += nw * 32)
            newton_job_group<P, REC, Q>(a, a.jobs2, base, count2, lane);
    }
    // last block (of every launch sharing the ticket): publish every problem's
    // step statistics (if asked), clear the job lists
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = a.nblocks > 0 ? (unsigned)a.nblocks : gridDim.x;
        __threadfence();
        last = atomicAdd(a.ticket, 1u) == total - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (a.publish) {
            const int nwb = blockDim.x >> 5, w = threadIdx.x >> 5;
            if (a.nprob <= nwb) {
                // few problems: a warp each, one stripe per lane
                if (w < a.nprob) publish_stats_warp(&a.stats[a.probs[w].stats], &a.probs[w], threadIdx.x & 31);
            } else {
                for (int p = threadIdx.x; p < a.nprob; p += blockDim.x)
                    publish_stats(&a.stats[a.probs[p].stats], &a.probs[p]);
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            *a.job_count = 0u;
            if (a.cursor) *a.cursor = 0u;
            if (a.job_count2) *a.job_count2 = 0u;
            *a.ticket = 0u;
        }
    }
}

template <typename P, bool REC>
static cudaError_t launch_t(const StepArgs& a, int grid, cudaStream_t s)
{
    d2q9_step_kernel<P, REC><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    return cudaGetLastError();
}

int d2q9_segment_width(int precision) { return precision == 1 ? 32 * Vd<float>::N : 32 * Vd<double>::N; }

cudaError_t launch_d2q9_step(int precision, const StepArgs& a, int grid, cudaStream_t s)
{
    if (grid <= 0) return cudaErrorInvalidValue;
    if (precision == 1) return a.rec ? launch_t<float, true>(a, grid, s) : launch_t<float, false>(a, grid, s);
    return a.rec ? launch_t<double, true>(a, grid, s) : launch_t<double, false>(a, grid, s);
}

cudaError_t launch_d2q9_tma(const StepArgs& a, const TmaMaps& m, cudaStream_t s)
{
    const int grid = m.nsegs * m.nparts;
    if (grid <= 0) return cudaErrorInvalidValue;
    if (a.rec) d2q9_tma_kernel<true><<<grid, kTmaThreads, 0, s>>>(a, m);
    else d2q9_tma_kernel<false><<<grid, kTmaThreads, 0, s>>>(a, m);
    return cudaGetLastError();
}

cudaError_t launch_d2q9_flat(const StepArgs& a, int nftiles, int nwrows, int ncblocks, int method, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // the nodes on or next to a wall (few), then rows 1 .. ny-2 of every strip
    const int nrb = std::min((nwrows + 7) / 8, sms * 4);
    if (nrb > 0) {
        if (a.rec) d2q9_wall_kernel<true><<<nrb, 256, 0, s>>>(a);
        else d2q9_wall_kernel<false><<<nrb, 256, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ncblocks > 0) {
        if (a.rec) d2q9_wall_cols_kernel<true><<<ncblocks, 256, 0, s>>>(a);
        else d2q9_wall_cols_kernel<false><<<ncblocks, 256, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nftiles > 0) {
        if (method == 1) {
            if (a.rec) d2q9_flat_kernel<true, true><<<nftiles, 256, 0, s>>>(a);
            else d2q9_flat_kernel<false, true><<<nftiles, 256, 0, s>>>(a);
        } else {
            if (a.rec) d2q9_flat_kernel<true, false><<<nftiles, 256, 0, s>>>(a);
            else d2q9_flat_kernel<false, false><<<nftiles, 256, 0, s>>>(a);
        }
        e = cudaGetLastError();
    }
    return e;
}

int d2q9_tma_blocks_per_sm()
{
    // all of the unified L1 / shared memory as shared memory: five blocks per SM
    cudaFuncSetAttribute(d2q9_tma_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(d2q9_tma_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_tma_kernel<false>, kTmaThreads, 0);
    return n > 0 ? n : 1;
}

template <int Q>
static cudaError_t launch_jobs_q(int precision, const JobArgs& a, int grid, cudaStream_t s, int prio, int threads)
{
    void (*k)(JobArgs) = precision == 1
                             ? (a.rec ? newton_jobs_kernel<float, true, Q> : newton_jobs_kernel<float, false, Q>)
                             : (a.rec ? newton_jobs_kernel<double, true, Q> : newton_jobs_kernel<double, false, Q>);
    // an explicit scheduling priority is a launch attribute, which a graph
    // captured from the stream keeps per kernel node
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = prio != 0 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, a);
}

cudaError_t launch_newton_jobs(int precision, int q, const JobArgs& a, cudaStream_t s, int grid, int prio, bool side)
{
    const int threads = side ? kJobSideThreads : kJobThreads;
    if (grid <= 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = sms * 2;
    }
    if (q == 9) return launch_jobs_q<9>(precision, a, grid, s, prio, threads);
    if (q == 5) return launch_jobs_q<5>(precision, a, grid, s, prio, threads);
    return cudaErrorInvalidValue;
}

int d2q9_blocks_per_sm(int precision)
{
    int n = 0;
    if (precision == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_step_kernel<float, false>, kWarpsPerBlock * 32, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_step_kernel<double, false>, kWarpsPerBlock * 32, 0);
    return n > 0 ? n : 1;
}

}  // namespace lbm
