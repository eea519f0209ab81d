// State initialization and field extraction.
//  * init: f_i = w_i theta0 (equilibrium, so Omega_i = w_i theta0), with nodes on
//    a Dirichlet wall set to the wall value; accumulates E(0).
//  * fields: theta = M0(f) = sum_i Omega_i, phi(theta), H = theta + phi/Ste (Sec. 2).
#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ bool dirichlet_value(const Problem& pb, int x, int y, double& td)
{
    const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) |
                      (pb.q == 9 ? ((y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0)) : 0);
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            td = pb.wall_theta[k];
            return true;
        }
    return false;
}

__device__ __forceinline__ double lat_w(int q, int i) { return q == 9 ? d2_w(i) : d1_w(i); }

template <typename P>
__global__ void init_state_kernel(const Problem* dprob, const double* __restrict__ theta0, int parity, DevStats* st)
{
    const Problem& pb = *dprob;
    P* s = static_cast<P*>(pb.state[parity]);
    const long long n = (long long)pb.nx * pb.ny;
    double e = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        double th = theta0[k], td;
        if (dirichlet_value(pb, x, y, td)) th = td;
        for (int i = 0; i < pb.q; ++i) s[i * pb.plane + (long long)(y + 1) * pb.pitch + x] = (P)(lat_w(pb.q, i) * th);
        e += th + phi_of(th, pb.inv_delta) * pb.inv_ste;
    }
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) acc_add(&st->cur_energy, e);
}

__global__ void wall_constants_kernel(Problem* probs, int nprob)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    Problem& pb = probs[p];
    for (int k = 0; k < 4; ++k) {
        const double t = tanh(pb.wall_theta[k] * pb.inv_delta);
        pb.wall_tanh[k] = t;
        pb.wall_phi[k] = 0.5 + 0.5 * t;
        pb.wall_th_hi[k] = (float)pb.wall_theta[k];
        pb.wall_th_lo[k] = (float)(pb.wall_theta[k] - (double)pb.wall_th_hi[k]);
        pb.wall_slope[k] = (float)(0.5 * (1.0 - t) * (1.0 + t) * pb.inv_delta * pb.inv_ste);
    }
    pb.wall_dth_max = (float)(1e-4 * pb.delta);
}

cudaError_t launch_wall_constants(Problem* dprobs, int nprob, cudaStream_t s)
{
    wall_constants_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob);
    return cudaGetLastError();
}

__global__ void finalize_init_kernel(DevStats* st)
{
    st->energy = acc_read(&st->cur_energy);
    st->energy_prev = st->energy;
    acc_clear(&st->cur_energy);
    st->have_energy = 1;
}

template <typename P>
__global__ void fields_kernel(const Problem* dprob, int parity, double* theta, double* phi, double* H,
                              double* theta_plane)
{
    const Problem& pb = *dprob;
    const P* s = static_cast<const P*>(pb.state[parity]);
    const long long n = (long long)pb.nx * pb.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        double th = 0.0;
        for (int i = pb.q - 1; i >= 0; --i) th += (double)s[i * pb.plane + (long long)(y + 1) * pb.pitch + x];
        const double ph = phi_of(th, pb.inv_delta);
        if (theta) theta[k] = th;
        if (phi) phi[k] = ph;
        if (H) H[k] = th + ph * pb.inv_ste;
        if (theta_plane) theta_plane[(long long)y * pb.pitch + x] = th;
    }
}

static int grid_for(long long n) { return (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16); }

cudaError_t launch_init_state(int precision, const Problem* dprob, const Problem& hp, const double* theta0,
                              int parity, DevStats* st, cudaStream_t s)
{
    const int g = grid_for((long long)hp.nx * hp.ny);
    if (precision == 1) init_state_kernel<float><<<g, 256, 0, s>>>(dprob, theta0, parity, st);
    else init_state_kernel<double><<<g, 256, 0, s>>>(dprob, theta0, parity, st);
    return cudaGetLastError();
}

cudaError_t launch_finalize_init(DevStats* st, cudaStream_t s)
{
    finalize_init_kernel<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_fields(int precision, const Problem* dprob, const Problem& hp, int parity, double* theta,
                          double* phi, double* H, double* theta_plane, cudaStream_t s)
{
    const int g = grid_for((long long)hp.nx * hp.ny);
    if (precision == 1) fields_kernel<float><<<g, 256, 0, s>>>(dprob, parity, theta, phi, H, theta_plane);
    else fields_kernel<double><<<g, 256, 0, s>>>(dprob, parity, theta, phi, H, theta_plane);
    return cudaGetLastError();
}

}  // namespace lbm
