// ILFBM step (Algorithm 1, the implicit liquid fraction based method of
// Sec. 3.3), the paper's second comparison scheme, in FP64: D1Q3 in one
// block (below), D2Q9 and D2Q5 with one launch per inner iteration (at the end).
//
// State: f_i (planes 0..q-1, theta = M0(f)) and the liquid fraction l (plane
// q of the same buffer).  One step:
//   theta = M0(f); l^(0) = l; for k = 1, 2, ...:
//     Omega_i = f_i - (f_i - w_i theta)/tau + (w_i/Ste)(l - l^(k-1))
//     f^(k)_i(y) = Omega_i(y - e_i), closures on the unknown one at a wall
//     H^(k) = M0(f^(k)) + l^(k-1)/Ste,  l^(k) = l(H^(k))  (lever rule)
//   until max_y |l^(k) - l^(k-1)| <= tol (at most maxit iterations; the
//   limit sets LBM_ERR_NEWTON); f~ = f^(k), l~ = l^(k).
// Closures: Dirichlet makes M0(f^(k)) = theta_D through the one unknown,
// bounce-back as for IREBM; a Dirichlet node's liquid fraction is that of its
// wall value, [theta_D > 0].
//
// Every inner iteration streams the whole lattice, and the loop's test is a
// maximum over the lattice, so the iterations of a step are separated by
// lattice-wide barriers.  D1Q3: a lattice of the paper's sizes (N <= 1601) fits
// in one thread block's shared memory (72 bytes per node): one block runs
// all steps of a call, its barriers are __syncthreads, and HBM is touched
// only at the start and the end of the call.  The inner loop is bound by the
// block's FP64 issue rate (FP64 is scarce on this GPU), so it is cut to what
// changes between iterations: the source-free part of the collision is formed
// once per step, an iteration forms only H^(k) and l^(k) (the populations
// f^(k) are streamed once, after the loop), and the loop's test is one flag
// per iteration behind a single barrier (three flags in rotation: the one
// cleared for the next iteration was last read two iterations earlier).
#include "lbm_device.cuh"

namespace lbm {

constexpr int kIlfThreads = 512;
constexpr int kIlfWarps = kIlfThreads / 32;

__device__ __forceinline__ double ilf_lever(double H, double ste, double inv_ste)
{
    return H < 0.0 ? 0.0 : (H > inv_ste ? 1.0 : ste * H);
}

__global__ void __launch_bounds__(kIlfThreads) ilfbm_d1q3_kernel(StepArgs a, int nsteps)
{
    extern __shared__ double sm[];
    __shared__ double red_e[2][kIlfWarps], red_f[2][kIlfWarps];   // per-step partial sums, step parity
    __shared__ int s_more[3];   // "some node changed by more than tol", iteration gk uses gk % 3
    const Problem& pb = a.probs[0];
    DevStats* st = &a.stats[pb.stats];
    const int n = pb.nx;
    double* o = sm;              // f_i at time t, then Omega_i without the source: f_i - (f_i - w_i theta)/tau
    double* fn = sm + 3 * n;     // f~ of the step (the buffers swap roles every step)
    double* el = sm + 6 * n;     // l at time t
    double* lb[2] = {el + n, el + 2 * n};   // l^(k-1) and l^(k), alternating
    const long long pl = pb.plane, row = pb.pitch;
    const double* src = static_cast<const double*>(pb.state[a.parity]);
    // the state at time t: f_i and l
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        for (int i = 0; i < 3; ++i) o[i * n + x] = src[i * pl + row + x];
        el[x] = src[3 * pl + row + x];
    }
    const double om = pb.omega, ste = pb.ste, inv_ste = pb.inv_ste, tol = pb.tol;
    const double w0 = d1_w(0), w1 = d1_w(1), w2 = d1_w(2);
    const double c0 = w0 * inv_ste, c1 = w1 * inv_ste, c2 = w2 * inv_ste;
    const bool dirW = pb.wall_kind[0] == 1, dirE = pb.wall_kind[1] == 1;
    const double thW = pb.wall_theta[0], thE = pb.wall_theta[1];
    const bool mirror = pb.bb_mode == 0;
    bool failed = false;
    unsigned gk = 0;   // inner iterations so far in this launch: selects the flag
    // thread 0: the statistics carried across the steps of this launch
    double E = 0.0, E_prev = 0.0, imb = 0.0, imb_max = 0.0, flux = 0.0;
    int have = 0, last_it = 0;
    if (threadIdx.x == 0) {
        E = st->energy;
        E_prev = st->energy_prev;
        imb = st->imbalance;
        imb_max = st->imbalance_max;
        flux = st->flux;
        have = st->have_energy;
        last_it = st->newton_max_iter;
    }
    if (threadIdx.x < 3) s_more[threadIdx.x] = 0;
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        // moments and the source-free part of the collision (the same in every
        // inner iteration); l^(0) = l
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const double f0 = o[x], f1 = o[n + x], f2 = o[2 * n + x];
            const double th = f0 + f1 + f2;
            o[x] = f0 - (f0 - w0 * th) * om;
            o[n + x] = f1 - (f1 - w1 * th) * om;
            o[2 * n + x] = f2 - (f2 - w2 * th) * om;
            lb[0][x] = el[x];
        }
        __syncthreads();
        // streamed f^(k)(y) from Omega_i(x) = o_i(x) + (w_i/Ste)(l(x) - l^(k-1)(x)),
        // the closures on the unknown one at a wall; returns the three values
        auto stream = [&](int y, const double* lp, double& q0, double& q1, double& q2) {
            q0 = o[y] + c0 * (el[y] - lp[y]);
            q1 = y > 0 ? o[n + y - 1] + c1 * (el[y - 1] - lp[y - 1]) : 0.0;
            q2 = y < n - 1 ? o[2 * n + y + 1] + c2 * (el[y + 1] - lp[y + 1]) : 0.0;
            if (y == 0)   // west wall: f_1 (e = +1) is unknown
                q1 = dirW ? thW - q0 - q2 : (mirror ? q2 : o[2 * n] + c2 * (el[0] - lp[0]));
            if (y == n - 1)   // east wall: f_2 (e = -1) is unknown
                q2 = dirE ? thE - q0 - q1 : (mirror ? q1 : o[n + n - 1] + c1 * (el[n - 1] - lp[n - 1]));
        };
        int it = 0, cur = 0;
        bool conv = false;
        while (!conv && it < pb.maxit) {   // it, gk, cur and conv are the same in every thread
            const double* lp = lb[cur];
            double* ln = lb[cur ^ 1];
            const int slot = gk % 3;
            ++it;
            ++gk;
            // H^(k) = M0(f^(k)) + l^(k-1)/Ste and the lever rule; Dirichlet nodes keep
            // the phase of their wall value
            bool more = false;
            for (int y = threadIdx.x; y < n; y += blockDim.x) {
                double lk;
                if (y == 0 && dirW) {
                    lk = thW > 0.0 ? 1.0 : 0.0;
                } else if (y == n - 1 && dirE) {
                    lk = thE > 0.0 ? 1.0 : 0.0;
                } else {
                    double q0, q1, q2;
                    stream(y, lp, q0, q1, q2);
                    lk = ilf_lever(q0 + q1 + q2 + lp[y] * inv_ste, ste, inv_ste);
                }
                more |= fabs(lk - lp[y]) > tol;
                ln[y] = lk;
            }
            // flag of this iteration; thread 0 clears the next iteration's flag, last read
            // two iterations ago (every thread read it before the previous barrier) and
            // next set after this iteration's barrier
            if (more) s_more[slot] = 1;
            if (threadIdx.x == 0) s_more[(slot + 1) % 3] = 0;
            __syncthreads();
            conv = s_more[slot] == 0;
            cur ^= 1;
        }
        failed |= !conv;
        // f~ = f^(k) (streamed with the source of l^(k-1)) into the other buffer,
        // l~ = l^(k); the boundary flux is filled minus leaving at the two walls
        const double* lp = lb[cur ^ 1];
        const double* ln = lb[cur];
        double e = 0.0, fl = 0.0;
        for (int y = threadIdx.x; y < n; y += blockDim.x) {
            double q0, q1, q2;
            stream(y, lp, q0, q1, q2);
            if (y == 0) fl += q1 - (o[2 * n] + c2 * (el[0] - lp[0]));
            if (y == n - 1) fl += q2 - (o[n + n - 1] + c1 * (el[n - 1] - lp[n - 1]));
            fn[y] = q0;
            fn[n + y] = q1;
            fn[2 * n + y] = q2;
            e += (q0 + q1 + q2) + ln[y] * inv_ste;
        }
        e = warp_sum(e);
        fl = warp_sum(fl);
        const int h = s & 1;
        if ((threadIdx.x & 31) == 0) {
            red_e[h][threadIdx.x >> 5] = e;
            red_f[h][threadIdx.x >> 5] = fl;
        }
        __syncthreads();   // every read of o, el and l^(k-1) of this step is done
        for (int y = threadIdx.x; y < n; y += blockDim.x) el[y] = ln[y];
        double* t = o;
        o = fn;
        fn = t;
        if (threadIdx.x == 0) {
            // the warps' sums in a fixed order; a half of red_* is written again two
            // steps later, after the next step's barriers, which thread 0 reaches
            // only after this
            double es = 0.0, fs = 0.0;
            for (int k = 0; k < kIlfWarps; ++k) {
                es += red_e[h][k];
                fs += red_f[h][k];
            }
            if (have) {
                imb = es - E - fs;
                if (fabs(imb) > imb_max) imb_max = fabs(imb);
            }
            E_prev = E;
            E = es;
            flux = fs;
            have = 1;
            last_it = it;
        }
    }
    if (threadIdx.x == 0) {
        st->energy = E;
        st->energy_prev = E_prev;
        st->imbalance = imb;
        st->imbalance_max = imb_max;
        st->flux = flux;
        st->have_energy = have;
        st->steps += nsteps;
        st->newton_nodes = 0;
        st->newton_max_iter = last_it;   // inner iterations of the last step
    }
    if (failed && threadIdx.x == 0) atomicOr(&st->error, 3);   // LBM_ERR_NEWTON: inner loop at its limit
    double* dst = static_cast<double*>(pb.state[a.parity ^ (nsteps & 1)]);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        for (int i = 0; i < 3; ++i) dst[i * pl + row + x] = o[i * n + x];
        dst[3 * pl + row + x] = el[x];
    }
}

// ---------------------------------------------------------------- 2D lattices
// ILFBM on D2Q9 and D2Q5 (Q = 9 or 5; the D2Q5 velocities are D2Q9's first
// five), FP64.  The inner loop needs a lattice-wide barrier per iteration, so
// an iteration is one launch; a step is
//   ilf2_collide   Omega0_i = f_i - (f_i - w_i theta)/tau in place, l^(0) = l
//   ilf2_s0        S0(y) = sum_i Omega0_i(y - e_i) at the interior nodes
//   ilf2_iter x maxit
//                  l^(k)(y) = l(H^(k)(y)), H^(k) = S0(y) + sum_i (w_i/Ste)
//                  (l - l^(k-1))(y - e_i) + l^(k-1)(y)/Ste at interior nodes, the
//                  closed streamed populations at wall nodes; a "changed" flag
//                  per iteration (three in rotation: launch k reads k-1's,
//                  sets its own and clears k+1's, last read by launch k-1); the
//                  first launch that finds the previous iteration unchanged
//                  records it and every later launch returns at once
//   ilf2_final     f~_i(y) = Omega_i(y - e_i) with the source of l^(K-1) and
//                  the closures, l~ = l^(K); energy sum theta~ + l~/Ste, flux,
//                  iteration count, the iteration-limit error; publishes
// Scratch (nx*ny doubles each): S0, l^(k) x 2, l - l^(k) x 2 (the interior
// stencil reads the differences, so an iteration spends one FMA per velocity).
// Node indices stay below 2^31 (the library's size limit), so the column and
// row come from a 32-bit division.
struct Ilf2Args {
    Problem pb;              // by value: the kernels read it from the parameter bank,
                             // so no store of theirs can alias it
    int parity;              // state[parity] holds f, then Omega0; f~ goes to state[parity ^ 1]
    double* s0;
    double* lb[2];           // l^(k-1) / l^(k) of iteration k: lb[(k-1) & 1] / lb[k & 1]
    double* dl[2];           // l - l^(k-1) / l - l^(k), written beside lb: the stencil's input
    unsigned int* flags;     // [0] done, [1] converged iteration, [2..4] changed per iteration mod 3
    DevStats* stats;
    unsigned int* ticket;
};

template <int Q>
__device__ __forceinline__ bool ilf2_known(const Problem& pb, int x, int y, int i)
{
    const int sx = x - d2_ex(i), sy = y - d2_ey(i);
    return sx >= 0 && sx < pb.nx && sy >= 0 && sy < pb.ny;
}

__device__ __forceinline__ int ilf2_dirichlet(const Problem& pb, int x, int y)
{
    const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0);
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) return k;
    return -1;
}

// Omega_i at node (x, y) with the source of the iterate lp: Omega0_i + (w_i/Ste)(l - lp)
template <int Q>
__device__ __forceinline__ double ilf2_omega(const Problem& pb, const double* st, const double* lp, int i, int x, int y)
{
    const long long nd = (long long)y * pb.nx + x;
    const double* lq = st + Q * pb.plane;
    return st[i * pb.plane + (long long)(y + 1) * pb.pitch + x] +
           lat_w(Q, i) * pb.inv_ste * (lq[(long long)(y + 1) * pb.pitch + x] - lp[nd]);
}

// the streamed populations of node (x, y) with the source of lp, closed at a wall
// (Dirichlet: the unknowns share theta_D - sum(known) by weight; bounce-back:
// mirror where the opposite is known, else link-wise); returns the flux term
// (filled minus leaving) when `flux` is set
template <int Q>
__device__ __forceinline__ double ilf2_streamed(const Problem& pb, const double* st, const double* lp, int x, int y,
                                                double (&q)[Q], bool flux)
{
    unsigned unk = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (ilf2_known<Q>(pb, x, y, i)) q[i] = ilf2_omega<Q>(pb, st, lp, i, x - d2_ex(i), y - d2_ey(i));
        else { q[i] = 0.0; unk |= 1u << i; }
    }
    if (!unk) return 0.0;
    const int wk = ilf2_dirichlet(pb, x, y);
    double in = 0.0, out = 0.0;
    if (wk >= 0) {
        double rest = pb.wall_theta[wk], wu = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if ((unk >> i) & 1) wu += lat_w(Q, i);
            else rest -= q[i];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((unk >> i) & 1) q[i] = lat_w(Q, i) * rest / wu;
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((unk >> i) & 1) {
                const int o = d2_opp(i);
                q[i] = (pb.bb_mode == 0 && !((unk >> o) & 1)) ? q[o] : ilf2_omega<Q>(pb, st, lp, o, x, y);
            }
    }
    if (flux) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((unk >> i) & 1) {
                in += q[i];
                out += ilf2_omega<Q>(pb, st, lp, d2_opp(i), x, y);   // Omega leaving through the wall
            }
    }
    return in - out;
}

template <int Q>
__global__ void __launch_bounds__(256) ilf2_collide(Ilf2Args a)
{
    const Problem& pb = a.pb;
    double* st = static_cast<double*>(pb.state[a.parity]);
    const long long n = (long long)pb.nx * pb.ny;
    if (blockIdx.x == 0 && threadIdx.x < 5) a.flags[threadIdx.x] = 0u;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)((unsigned)k % (unsigned)pb.nx), y = (int)((unsigned)k / (unsigned)pb.nx);
        const long long at = (long long)(y + 1) * pb.pitch + x;
        double f[Q], th = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = st[i * pb.plane + at];
            th += f[i];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) st[i * pb.plane + at] = f[i] - (f[i] - lat_w(Q, i) * th) * pb.omega;
        a.lb[0][k] = st[Q * pb.plane + at];
        a.dl[0][k] = 0.0;   // l - l^(0)
    }
}

template <int Q>
__global__ void __launch_bounds__(256) ilf2_s0(Ilf2Args a)
{
    const Problem& pb = a.pb;
    const double* st = static_cast<const double*>(pb.state[a.parity]);
    const long long n = (long long)pb.nx * pb.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)((unsigned)k % (unsigned)pb.nx), y = (int)((unsigned)k / (unsigned)pb.nx);
        if (x == 0 || x == pb.nx - 1 || y == 0 || y == pb.ny - 1) continue;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            s += st[i * pb.plane + (long long)(y - d2_ey(i) + 1) * pb.pitch + x - d2_ex(i)];
        a.s0[k] = s;
    }
}

template <int Q>
__global__ void __launch_bounds__(256) ilf2_iter(Ilf2Args a, int k)
{
    volatile unsigned int* fl = a.flags;
    if (fl[0]) return;   // converged in an earlier iteration
    if (k > 1 && fl[2 + (k - 1) % 3] == 0u) {
        // iteration k - 1 changed nothing: it is the last one
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            fl[1] = (unsigned)(k - 1);
            fl[0] = 1u;
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) fl[2 + (k + 1) % 3] = 0u;
    const Problem& pb = a.pb;
    const double* st = static_cast<const double*>(pb.state[a.parity]);
    const double* lq = st + Q * pb.plane;
    const double* lp = a.lb[(k - 1) & 1];
    const double* dp = a.dl[(k - 1) & 1];
    double* ln = a.lb[k & 1];
    double* dn = a.dl[k & 1];
    const long long n = (long long)pb.nx * pb.ny;
    bool more = false;
    for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n; nd += (long long)gridDim.x * blockDim.x) {
        const int x = (int)((unsigned)nd % (unsigned)pb.nx), y = (int)((unsigned)nd / (unsigned)pb.nx);
        const int wk = ilf2_dirichlet(pb, x, y);
        double lk;
        if (wk >= 0) {
            lk = pb.wall_theta[wk] > 0.0 ? 1.0 : 0.0;
        } else {
            double H;
            if (x > 0 && x < pb.nx - 1 && y > 0 && y < pb.ny - 1) {
                H = a.s0[nd];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const long long sn = (long long)(y - d2_ey(i)) * pb.nx + x - d2_ex(i);
                    H += lat_w(Q, i) * pb.inv_ste * dp[sn];
                }
            } else {
                double q[Q];
                (void)ilf2_streamed<Q>(pb, st, lp, x, y, q, false);
                H = 0.0;
#pragma unroll
                for (int i = 0; i < Q; ++i) H += q[i];
            }
            H += lp[nd] * pb.inv_ste;
            lk = ilf_lever(H, pb.ste, pb.inv_ste);
        }
        more |= fabs(lk - lp[nd]) > pb.tol;
        ln[nd] = lk;
        dn[nd] = lq[(long long)(y + 1) * pb.pitch + x] - lk;
    }
    if (__any_sync(kFull, more) && (threadIdx.x & 31) == 0) fl[2 + k % 3] = 1u;
}

template <int Q>
__global__ void __launch_bounds__(256) ilf2_final(Ilf2Args a, int maxit)
{
    const Problem& pb = a.pb;
    const volatile unsigned int* fl = a.flags;
    const bool done = fl[0] != 0u;
    const int K = done ? (int)fl[1] : maxit;
    const bool conv = done || fl[2 + maxit % 3] == 0u;
    const double* st = static_cast<const double*>(pb.state[a.parity]);
    double* dst = static_cast<double*>(pb.state[a.parity ^ 1]);
    const double* lp = a.lb[(K - 1) & 1];
    const double* ln = a.lb[K & 1];
    DevStats* sts = &a.stats[pb.stats];
    const long long n = (long long)pb.nx * pb.ny;
    double e = 0.0, fx = 0.0;
    for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < n; nd += (long long)gridDim.x * blockDim.x) {
        const int x = (int)((unsigned)nd % (unsigned)pb.nx), y = (int)((unsigned)nd / (unsigned)pb.nx);
        double q[Q];
        fx += ilf2_streamed<Q>(pb, st, lp, x, y, q, true);
        const long long at = (long long)(y + 1) * pb.pitch + x;
        double th = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            dst[i * pb.plane + at] = q[i];
            th += q[i];
        }
        dst[Q * pb.plane + at] = ln[nd];
        e += th + ln[nd] * pb.inv_ste;
    }
    e = warp_sum(e);
    fx = warp_sum(fx);
    if ((threadIdx.x & 31) == 0) {
        acc_add(&my_stripe(sts)->energy, e);
        acc_add(&my_stripe(sts)->flux, fx);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicMax(&sts->cur_maxit, K);
        if (!conv) atomicOr(&sts->error, 3);   // LBM_ERR_NEWTON: the inner loop reached its limit
    }
    finish_launch(a.stats, 1, a.ticket);
}

template <int Q>
static cudaError_t ilf2_step(const Ilf2Args& a, int maxit, int grid, cudaStream_t s)
{
    ilf2_collide<Q><<<grid, 256, 0, s>>>(a);
    ilf2_s0<Q><<<grid, 256, 0, s>>>(a);
    for (int k = 1; k <= maxit; ++k) ilf2_iter<Q><<<grid, 256, 0, s>>>(a, k);
    ilf2_final<Q><<<grid, 256, 0, s>>>(a, maxit);
    return cudaGetLastError();
}

cudaError_t launch_ilfbm_2d(const Problem& hp, int parity, double* scratch,
                            unsigned int* flags, DevStats* stats, unsigned int* ticket, cudaStream_t s)
{
    Ilf2Args a;
    a.pb = hp;
    a.parity = parity;
    const long long n = (long long)hp.nx * hp.ny;
    a.s0 = scratch;
    a.lb[0] = scratch + n;
    a.lb[1] = scratch + 2 * n;
    a.dl[0] = scratch + 3 * n;
    a.dl[1] = scratch + 4 * n;
    a.flags = flags;
    a.stats = stats;
    a.ticket = ticket;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    return hp.q == 9 ? ilf2_step<9>(a, hp.maxit, grid, s) : ilf2_step<5>(a, hp.maxit, grid, s);
}

static size_t ilfbm_smem(int nx) { return (size_t)9 * nx * sizeof(double); }

bool ilfbm_d1q3_fits(int nx) { return ilfbm_smem(nx) <= 200 * 1024; }

cudaError_t launch_ilfbm_d1q3(const StepArgs& a, const Problem& hp, int nsteps, cudaStream_t s)
{
    const size_t sm = ilfbm_smem(hp.nx);
    cudaError_t e = cudaFuncSetAttribute(ilfbm_d1q3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ilfbm_d1q3_kernel<<<1, kIlfThreads, sm, s>>>(a, nsteps);
    return cudaGetLastError();
}

}  // namespace lbm
