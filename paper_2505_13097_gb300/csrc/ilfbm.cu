// ILFBM step (Algorithm 1, the implicit liquid fraction based method of
// Sec. 3.3), the paper's second comparison scheme, on D1Q3 in FP64.
//
// State: f_i (planes 0..2, theta = M0(f)) and the liquid fraction l (plane 3
// of the same buffer).  One step:
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
// lattice-wide barriers.  A 1D lattice of the paper's sizes (N <= 1601) fits
// in one thread block's shared memory (72 bytes per node): one block runs
// all steps of a call, its barriers are __syncthreads, and HBM is touched
// only at the start and the end of the call.
#include "lbm_device.cuh"

namespace lbm {

constexpr int kIlfThreads = 512;
constexpr int kIlfWarps = kIlfThreads / 32;

// Deterministic block reductions: warp shuffles, then a fixed order over warps.
__device__ __forceinline__ double ilf_block_sum(double v, double* sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < kIlfWarps; ++k) s += sh[k];
    return s;   // the same value in every thread
}
__device__ __forceinline__ double ilf_block_max(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double m = 0.0;
    for (int k = 0; k < kIlfWarps; ++k) m = fmax(m, sh[k]);
    return m;
}

__device__ __forceinline__ double ilf_lever(double H, double ste, double inv_ste)
{
    return H < 0.0 ? 0.0 : (H > inv_ste ? 1.0 : ste * H);
}

__global__ void __launch_bounds__(kIlfThreads) ilfbm_d1q3_kernel(StepArgs a, int nsteps)
{
    extern __shared__ double sm[];
    __shared__ double red[kIlfWarps];
    __shared__ double s_flux[2];
    const Problem& pb = a.probs[0];
    DevStats* st = &a.stats[pb.stats];
    const int n = pb.nx;
    double* f = sm;              // f_i at time t, 3 n
    double* fk = f + 3 * n;      // inner iterate f^(k), 3 n
    double* th = fk + 3 * n;     // theta = M0(f)
    double* el = th + n;         // l at time t
    double* lp = el + n;         // l^(k-1), replaced by l^(k) at the end of an iteration
    const long long pl = pb.plane, row = pb.pitch;
    const double* src = static_cast<const double*>(pb.state[a.parity]);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        for (int i = 0; i < 3; ++i) f[i * n + x] = src[i * pl + row + x];
        el[x] = src[3 * pl + row + x];
    }
    const double om = pb.omega, ste = pb.ste, inv_ste = pb.inv_ste, tol = pb.tol;
    const double w[3] = {d1_w(0), d1_w(1), d1_w(2)};
    const bool dirW = pb.wall_kind[0] == 1, dirE = pb.wall_kind[1] == 1;
    const double thW = pb.wall_theta[0], thE = pb.wall_theta[1];
    bool failed = false;
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            th[x] = f[x] + f[n + x] + f[2 * n + x];
            lp[x] = el[x];
        }
        __syncthreads();
        // Omega_i at node x: collision with the source of the current iterate
        auto Om = [&](int i, int x) -> double {
            const double fi = f[i * n + x];
            return fi - (fi - w[i] * th[x]) * om + w[i] * inv_ste * (el[x] - lp[x]);
        };
        int it = 0;
        bool conv = false;
        while (!conv && it < pb.maxit) {   // it and conv are the same in every thread
            ++it;
            for (int y = threadIdx.x; y < n; y += blockDim.x) {
                const double q0 = Om(0, y);
                double q1 = y > 0 ? Om(1, y - 1) : 0.0;
                double q2 = y < n - 1 ? Om(2, y + 1) : 0.0;
                if (y == 0) {
                    // west wall: f_1 (e = +1) is unknown
                    q1 = dirW ? thW - q0 - q2 : (pb.bb_mode == 0 ? q2 : Om(2, 0));
                    s_flux[0] = q1 - Om(2, 0);
                }
                if (y == n - 1) {
                    // east wall: f_2 (e = -1) is unknown
                    q2 = dirE ? thE - q0 - q1 : (pb.bb_mode == 0 ? q1 : Om(1, n - 1));
                    s_flux[1] = q2 - Om(1, n - 1);
                }
                fk[y] = q0;
                fk[n + y] = q1;
                fk[2 * n + y] = q2;
            }
            __syncthreads();
            // enthalpy and lever rule; Dirichlet nodes keep the phase of their wall value
            double ch = 0.0;
            for (int y = threadIdx.x; y < n; y += blockDim.x) {
                double lk;
                if (y == 0 && dirW) lk = thW > 0.0 ? 1.0 : 0.0;
                else if (y == n - 1 && dirE) lk = thE > 0.0 ? 1.0 : 0.0;
                else lk = ilf_lever(fk[y] + fk[n + y] + fk[2 * n + y] + lp[y] * inv_ste, ste, inv_ste);
                ch = fmax(ch, fabs(lk - lp[y]));
                lp[y] = lk;
            }
            conv = ilf_block_max(ch, red) <= tol;   // ends with a barrier before lp is read again
        }
        failed |= !conv;
        double e = 0.0;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const double a0 = fk[x], a1 = fk[n + x], a2 = fk[2 * n + x];
            f[x] = a0;
            f[n + x] = a1;
            f[2 * n + x] = a2;
            el[x] = lp[x];
            e += (a0 + a1 + a2) + lp[x] * inv_ste;
        }
        const double es = ilf_block_sum(e, red);
        if (threadIdx.x == 0) {
            const double fl = s_flux[0] + s_flux[1];
            if (st->have_energy) {
                const double imb = es - st->energy - fl;
                st->imbalance = imb;
                if (fabs(imb) > st->imbalance_max) st->imbalance_max = fabs(imb);
            }
            st->energy_prev = st->energy;
            st->energy = es;
            st->flux = fl;
            st->have_energy = 1;
            st->steps += 1;
            st->newton_nodes = 0;
            st->newton_max_iter = it;   // inner iterations of this step
        }
        __syncthreads();
    }
    if (failed && threadIdx.x == 0) atomicOr(&st->error, 3);   // LBM_ERR_NEWTON: inner loop at its limit
    double* dst = static_cast<double*>(pb.state[a.parity ^ (nsteps & 1)]);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        for (int i = 0; i < 3; ++i) dst[i * pl + row + x] = f[i * n + x];
        dst[3 * pl + row + x] = el[x];
    }
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
