// D1Q3 IREBM step (Algorithm 3 on the 1D lattice of Sec. 3.2).
//
// Two kernels share the per-node update:
//  * d1q3_step_kernel: one thread per node, one launch per step (any size);
//  * d1q3_fused_kernel: one thread block keeps the whole lattice in shared
//    memory and runs many steps per launch, synchronizing the block between
//    steps.  A 512-node lattice is far too small to fill the GPU, so the
//    per-step cost is launch latency unless the steps are fused.
// Moments are summed in FP64 for both storage precisions (three terms).
// EEBM (Algorithm 2) runs in the same kernels (method 1 of the problem).
#include "lbm_device.cuh"

namespace lbm {

struct NodeOut {
    double theta_new;   // theta' of the node
    double energy;      // theta' + phi(theta')/Ste
    double flux;        // boundary flux contribution
    int newton;         // 1 if the Newton iteration ran
    int iters;
    bool fail;
};

// One node: u = Omega(x) at time t, ql/qr = Omega_1(x-1), Omega_2(x+1) (ignored at walls).
template <typename P>
__device__ __forceinline__ NodeOut d1q3_node(const Problem& pb, int x, const P (&u)[3], P ql, P qr, P (&o)[3])
{
    NodeOut r;
    r.flux = 0.0;
    r.newton = 0;
    r.iters = 0;
    r.fail = false;
    double q[3] = {(double)u[0], (double)ql, (double)qr};
    const double th = (double)u[0] + (double)u[1] + (double)u[2];
    bool dir = false;
    double thd = 0.0;
    const bool west = x == 0, east = x == pb.nx - 1;
    if (west || east) {
        // nx >= 2: the west node misses q_1 (e = +1), the east node q_2 (e = -1) (Sec. 4.2)
        const int side = west ? 0 : 1;
        const int iu = west ? 1 : 2, io = west ? 2 : 1;
        const double out = (double)u[io];   // Omega leaving through this wall
        if (pb.wall_kind[side] == 1) {
            dir = true;
            thd = pb.wall_theta[side];
            // Eq. (16): the single unknown closes M0(q), with M0(q) from Eq. (14) at theta' = theta_D
            // (EEBM: the wall value's enthalpy, Algorithm 2 keeps H = M0)
            const double m0t = pb.method == 1 ? pb.wall_H[side]
                                              : thd + (phi_of(thd, pb.inv_delta) - phi_of(th, pb.inv_delta)) * pb.inv_ste;
            q[iu] = (double)(P)(m0t - q[0] - q[io]);
        } else {
            // bounce-back q_iu = q_io (Sec. 4.2.2), or link-wise q_iu = Omega_io at the node
            q[iu] = pb.bb_mode == 0 ? q[io] : (double)u[io];
        }
        r.flux = q[iu] - out;
    }
    const double m0 = q[2] + q[1] + q[0];
    if (pb.method == 1) {
        // EEBM (Algorithm 2): H = M0(q), theta = Theta(H), relaxation toward
        // w_i theta (i != 0) and H - (1 - w_0) theta (i = 0); the energy is H
        const double H = m0, t = eebm_theta(H, pb.inv_ste), om = pb.omega, omc = 1.0 - pb.omega;
        o[0] = (P)(omc * q[0] + om * (H - (1.0 - d1_w(0)) * t));
        o[1] = (P)(omc * q[1] + om * d1_w(1) * t);
        o[2] = (P)(omc * q[2] + om * d1_w(2) * t);
        r.theta_new = t;
        r.energy = H;
        return r;
    }
    double tn, phn;
    if (dir) {
        tn = thd;
        phn = phi_of(thd, pb.inv_delta);
    } else {
        const double thr = kSat * pb.delta;
        if ((th >= thr && m0 >= thr) || (th <= -thr && m0 <= -thr)) {
            tn = m0;
            phn = m0 > 0.0 ? 1.0 : 0.0;
        } else {
            const double pth = phi_of(th, pb.inv_delta);
            NewtonOut nr = newton_mixed(m0, th, pth, pb);
            r.fail = !nr.ok || !isfinite(nr.root);
            tn = m0 + (pth - nr.phi_root) * pb.inv_ste;
            phn = nr.phi_root;
            r.newton = 1;
            r.iters = nr.iters;
        }
    }
    const double cc = tn - (1.0 - pb.omega) * m0;
    const double omc = 1.0 - pb.omega;
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = (P)(omc * q[i] + d1_w(i) * cc);
    r.theta_new = tn;
    r.energy = tn + phn * pb.inv_ste;
    return r;
}

template <typename P>
__global__ void __launch_bounds__(128) d1q3_step_kernel(StepArgs a)
{
    const Problem& pb = a.probs[0];
    DevStats* st = &a.stats[pb.stats];
    const P* src = static_cast<const P*>(pb.state[a.parity]);
    P* dst = static_cast<P*>(pb.state[a.parity ^ 1]);
    const long long pl = pb.plane, row = pb.pitch;   // row 0 of a plane starts at +pitch
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, f = 0.0;
    int nn = 0, mi = 0;
    if (x < pb.nx) {
        P u[3], o[3];
        for (int i = 0; i < 3; ++i) u[i] = src[i * pl + row + x];
        const P ql = x > 0 ? src[1 * pl + row + x - 1] : (P)0;
        const P qr = x < pb.nx - 1 ? src[2 * pl + row + x + 1] : (P)0;
        NodeOut r = d1q3_node<P>(pb, x, u, ql, qr, o);
        for (int i = 0; i < 3; ++i) dst[i * pl + row + x] = o[i];
        if (a.rec) a.rec[x] = r.theta_new;
        if (r.fail) atomicOr(&st->error, 3);
        e = r.energy;
        f = r.flux;
        nn = r.newton;
        mi = r.iters;
    }
    e = warp_sum(e);
    f = warp_sum(f);
    nn = warp_sum_i(nn);
    mi = warp_max_i(mi);
    if ((threadIdx.x & 31) == 0) {
        acc_add(&my_stripe(st)->energy, e);
        acc_add(&my_stripe(st)->flux, f);
        if (nn) atomicAdd(&my_stripe(st)->newton, (unsigned long long)nn);
        if (mi) atomicMax(&st->cur_maxit, mi);
    }
    finish_launch(a.stats, 1, a.ticket);
}

constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;

// One block keeps the lattice in shared memory and runs `nsteps` steps.  A
// step ends at a single barrier: the warps' partial sums go to a per-step
// parity half of a small array, and thread 0 sums them in a fixed warp order
// (deterministic) after the barrier while the others start the next step; a
// warp writes that half again only two steps later, after the next barrier,
// which thread 0 reaches only when it has read it.  Thread 0 keeps the
// statistics in registers and writes them once at the end.
template <typename P>
__global__ void __launch_bounds__(kFusedThreads) d1q3_fused_kernel(StepArgs a, int nsteps, double* rec)
{
    extern __shared__ unsigned char smem_raw[];
    const Problem& pb = a.probs[0];
    DevStats* st = &a.stats[pb.stats];
    const int n = pb.nx;
    P* buf[2] = {reinterpret_cast<P*>(smem_raw), reinterpret_cast<P*>(smem_raw) + 3 * n};
    __shared__ double red_e[2][kFusedWarps], red_f[2][kFusedWarps];
    __shared__ int red_n[2][kFusedWarps], red_m[2][kFusedWarps];
    const long long pl = pb.plane, row = pb.pitch;
    const P* src = static_cast<const P*>(pb.state[a.parity]);
    for (int x = threadIdx.x; x < n; x += blockDim.x)
        for (int i = 0; i < 3; ++i) buf[0][i * n + x] = src[i * pl + row + x];
    // thread 0: the statistics carried across the steps of this launch
    double E = 0.0, imb = 0.0, imb_max = 0.0, flux = 0.0, E_prev = 0.0;
    int have = 0, last_n = 0, last_m = 0;
    if (threadIdx.x == 0) {
        E = st->energy;
        E_prev = st->energy_prev;
        imb = st->imbalance;
        imb_max = st->imbalance_max;
        flux = st->flux;
        have = st->have_energy;
        last_n = (int)st->newton_nodes;
        last_m = st->newton_max_iter;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    bool fail = false;
    __syncthreads();
    int cur = 0;
    for (int s = 0; s < nsteps; ++s) {
        const P* in = buf[cur];
        P* out = buf[cur ^ 1];
        double e = 0.0, f = 0.0;
        int nn = 0, mi = 0;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            P u[3] = {in[x], in[n + x], in[2 * n + x]}, o[3];
            const P ql = x > 0 ? in[n + x - 1] : (P)0;
            const P qr = x < n - 1 ? in[2 * n + x + 1] : (P)0;
            NodeOut r = d1q3_node<P>(pb, x, u, ql, qr, o);
            out[x] = o[0];
            out[n + x] = o[1];
            out[2 * n + x] = o[2];
            if (rec) rec[(long long)s * pb.pitch + x] = r.theta_new;
            e += r.energy;
            f += r.flux;
            nn += r.newton;
            mi = max(mi, r.iters);
            fail |= r.fail;
        }
        e = warp_sum(e);
        f = warp_sum(f);
        nn = warp_sum_i(nn);
        mi = warp_max_i(mi);
        const int h = s & 1;
        if (l == 0) {
            red_e[h][w] = e;
            red_f[h][w] = f;
            red_n[h][w] = nn;
            red_m[h][w] = mi;
        }
        __syncthreads();   // the step's writes of `out` and of the partial sums are complete
        if (threadIdx.x == 0) {
            double es = 0.0, fs = 0.0;
            int nsum = 0, mmax = 0;
            for (int k = 0; k < kFusedWarps; ++k) {
                es += red_e[h][k];
                fs += red_f[h][k];
                nsum += red_n[h][k];
                mmax = max(mmax, red_m[h][k]);
            }
            if (have) {
                imb = es - E - fs;
                if (fabs(imb) > imb_max) imb_max = fabs(imb);
            }
            E_prev = E;
            E = es;
            flux = fs;
            have = 1;
            last_n = nsum;
            last_m = mmax;
        }
        cur ^= 1;
    }
    if (fail) atomicOr(&st->error, 3);
    if (threadIdx.x == 0) {
        st->energy = E;
        st->energy_prev = E_prev;
        st->imbalance = imb;
        st->imbalance_max = imb_max;
        st->flux = flux;
        st->have_energy = have;
        st->steps += nsteps;
        st->newton_nodes = last_n;
        st->newton_max_iter = last_m;
    }
    P* dst = static_cast<P*>(pb.state[a.parity ^ (nsteps & 1)]);
    for (int x = threadIdx.x; x < n; x += blockDim.x)
        for (int i = 0; i < 3; ++i) dst[i * pl + row + x] = buf[cur][i * n + x];
}

static size_t fused_smem(int precision, int nx) { return (size_t)2 * 3 * nx * (precision == 1 ? 4 : 8); }

bool d1q3_fused_fits(int precision, int nx) { return fused_smem(precision, nx) <= 200 * 1024; }

cudaError_t launch_d1q3_step(int precision, const StepArgs& a, const Problem& hp, cudaStream_t s)
{
    const int grid = (hp.nx + 127) / 128;
    if (precision == 1) d1q3_step_kernel<float><<<grid, 128, 0, s>>>(a);
    else d1q3_step_kernel<double><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_d1q3_fused(int precision, const StepArgs& a, const Problem& hp, int nsteps, int start_parity,
                              double* rec, cudaStream_t s)
{
    StepArgs b = a;
    b.parity = start_parity;
    const size_t sm = fused_smem(precision, hp.nx);
    cudaError_t e;
    if (precision == 1) {
        e = cudaFuncSetAttribute(d1q3_fused_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        d1q3_fused_kernel<float><<<1, kFusedThreads, sm, s>>>(b, nsteps, rec);
    } else {
        e = cudaFuncSetAttribute(d1q3_fused_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        d1q3_fused_kernel<double><<<1, kFusedThreads, sm, s>>>(b, nsteps, rec);
    }
    return cudaGetLastError();
}

}  // namespace lbm
