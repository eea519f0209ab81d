// State initialization and field extraction.
//  * init: f_i = w_i theta0 (equilibrium, so Omega_i = w_i theta0), with nodes on
//    a Dirichlet wall set to the wall value; accumulates E(0).  EEBM: the
//    equilibrium of H(theta0); ILFBM: also l = [theta0 > 0] in plane q.
//  * fields: theta = M0(f) = sum_i Omega_i, phi(theta), H = theta + phi/Ste (Sec. 2);
//    EEBM: theta = Theta(H); ILFBM: phi = l.
#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ bool dirichlet_value(const Problem& pb, int x, int y, double& td)
{
    const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) |
                      (pb.q != 3 ? ((y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0)) : 0);
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            td = pb.wall_theta[k];
            return true;
        }
    return false;
}

// The shift s of an FP32 state (its populations are stored less w_i s),
// written to the tail of both buffers: half the mean over the nodes of the
// initial M0 (theta0; EEBM: H(theta0)), rounded to a float.  A stored value's
// rounding error scales with its size, |M0 - s| w_i.  Storing Omega_i itself
// (s = 0) lets the rounding of a smooth field far from the front drift
// coherently (on the 4096^2 melting workload, 2.45e-5 of theta after 10,000
// steps against the FP64 form); s = the mean of M0 removes that but makes the
// values at the melting point (M0 = 0, where phi' is largest) the large ones
// (max |d phi| 1.04e-4).  Halfway between the two bounds both.  One block; a
// fixed summation order (deterministic).
__global__ void __launch_bounds__(1024) shift_kernel(const Problem* dprob, const double* __restrict__ theta0)
{
    __shared__ double part[1024];
    const Problem& pb = *dprob;
    const long long n = (long long)pb.nx * pb.ny;
    double v = 0.0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
        const double th = theta0[k];
        v += pb.method == 1 ? th + (th > 0.0 ? pb.inv_ste : 0.0) : th;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float sh = n > 0 ? (float)(0.5 * part[0] / (double)n) : 0.f;
        for (int b = 0; b < 2; ++b) *reinterpret_cast<float*>(static_cast<char*>(pb.state[b]) + pb.tail_off) = sh;
    }
}

template <typename P>
__global__ void init_state_kernel(const Problem* dprob, const double* __restrict__ theta0, int parity, DevStats* st)
{
    const Problem& pb = *dprob;
    P* s = static_cast<P*>(pb.state[parity]);
    // FP32: the populations are stored less w_i sh
    const double sh = sizeof(P) == 4 ? (double)state_shift(pb, parity) : 0.0;
    const long long n = (long long)pb.nx * pb.ny;
    double e = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        double th = theta0[k], td;
        if (dirichlet_value(pb, x, y, td)) th = td;
        if (pb.method == 1) {
            // EEBM: equilibrium of H = theta + [theta > 0]/Ste (Algorithm 2): w_i theta,
            // and H - (1 - w_0) theta for i = 0
            const double H = th + (th > 0.0 ? pb.inv_ste : 0.0);
            for (int i = 0; i < pb.q; ++i)
                s[i * pb.plane + (long long)(y + 1) * pb.pitch + x] =
                    (P)(i == 0 ? H - (1.0 - lat_w(pb.q, 0)) * th - lat_w(pb.q, 0) * sh : lat_w(pb.q, i) * (th - sh));
            e += H;
            continue;
        }
        for (int i = 0; i < pb.q; ++i)
            s[i * pb.plane + (long long)(y + 1) * pb.pitch + x] = (P)(lat_w(pb.q, i) * (th - sh));
        if (pb.method == 2) {
            // ILFBM (Algorithm 1): the liquid fraction of the initial phase, plane q
            const double l = th > 0.0 ? 1.0 : 0.0;
            s[pb.q * pb.plane + (long long)(y + 1) * pb.pitch + x] = (P)l;
            e += th + l * pb.inv_ste;
            continue;
        }
        e += th + phi_of(th, pb.inv_delta) * pb.inv_ste;
    }
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) acc_add(&my_stripe(st)->energy, e);
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
    for (int k = 0; k < 4; ++k) {
        pb.wall_H[k] = pb.wall_theta[k] + (pb.wall_theta[k] > 0.0 ? pb.inv_ste : 0.0);
        pb.wall_H_hi[k] = (float)pb.wall_H[k];
        pb.wall_H_lo[k] = (float)(pb.wall_H[k] - (double)pb.wall_H_hi[k]);
    }
}

cudaError_t launch_wall_constants(Problem* dprobs, int nprob, cudaStream_t s)
{
    wall_constants_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob);
    return cudaGetLastError();
}

__global__ void finalize_init_kernel(DevStats* st)
{
    AccSum esum = {{0ull, 0ull, 0ull, 0ull}};
    for (int k = 0; k < kStripes; ++k)
        for (int j = 0; j < 4; ++j) esum.limb[j] += st->cur[k].energy.limb[j];
    st->energy = acc_read(&esum);
    st->energy_prev = st->energy;
    for (int k = 0; k < kStripes; ++k) acc_clear(&st->cur[k].energy);
    st->have_energy = 1;
}

template <typename P>
__global__ void fields_kernel(const Problem* dprob, int parity, double* theta, double* phi, double* H,
                              double* theta_plane)
{
    const Problem& pb = *dprob;
    const P* s = static_cast<const P*>(pb.state[parity]);
    const double sh = sizeof(P) == 4 ? (double)state_shift(pb, parity) : 0.0;   // FP32: stored less w_i sh
    const long long n = (long long)pb.nx * pb.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        double th = sh;
        for (int i = pb.q - 1; i >= 0; --i) th += (double)s[i * pb.plane + (long long)(y + 1) * pb.pitch + x];
        if (pb.method == 1) {
            // EEBM: M0 is the enthalpy; theta = Theta(H), liquid fraction min(max(Ste H, 0), 1)
            const double h = th;
            th = eebm_theta(h, pb.inv_ste);
            if (theta) theta[k] = th;
            if (phi) phi[k] = fmin(fmax(h * pb.ste, 0.0), 1.0);
            if (H) H[k] = h;
            if (theta_plane) theta_plane[(long long)y * pb.pitch + x] = th;
            continue;
        }
        // ILFBM: the liquid fraction is a field of its own (plane q)
        const double ph = pb.method == 2 ? (double)s[pb.q * pb.plane + (long long)(y + 1) * pb.pitch + x]
                                         : phi_of(th, pb.inv_delta);
        if (theta) theta[k] = th;
        if (phi) phi[k] = ph;
        if (H) H[k] = th + ph * pb.inv_ste;
        if (theta_plane) theta_plane[(long long)y * pb.pitch + x] = th;
    }
}

// Interface position along the lattice lines that start at `wall` (0 W, 1 E,
// 2 S, 3 N; node 0 on the wall), one warp per line: the first sign change of
// theta = M0(f) from the wall node's sign, linearly interpolated (node units;
// 0 if theta is 0 on the wall node, n - 1 if the sign never changes), and the
// wall side's phase fraction summed along the line minus the wall half cell.
// out[line] and out[nlines + line].
template <typename P>
__global__ void front_kernel(const Problem* dprob, int parity, int wall, double* out)
{
    const Problem& pb = *dprob;
    const P* s = static_cast<const P*>(pb.state[parity]);
    const bool rows = wall <= 1;
    const int nlines = rows ? pb.ny : pb.nx;
    const int n = rows ? pb.nx : pb.ny;
    const double sh = sizeof(P) == 4 ? (double)state_shift(pb, parity) : 0.0;   // FP32: stored less w_i sh
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int line = w0; line < nlines; line += nw) {
        auto theta_at = [&](int i) -> double {
            int x, y;
            if (wall == 0) { x = i; y = line; }
            else if (wall == 1) { x = pb.nx - 1 - i; y = line; }
            else if (wall == 2) { x = line; y = i; }
            else { x = line; y = pb.ny - 1 - i; }
            double th = sh;
            for (int k = pb.q - 1; k >= 0; --k) th += (double)s[k * pb.plane + (long long)(y + 1) * pb.pitch + x];
            return pb.method == 1 ? eebm_theta(th, pb.inv_ste) : th;
        };
        const double t0 = __shfl_sync(kFull, lane == 0 ? theta_at(0) : 0.0, 0);
        const bool hot = t0 > 0.0;
        double fz = t0 == 0.0 ? 0.0 : -1.0;   // -1: not found yet
        double prev_last = t0;                // theta of the node before this chunk
        double sum = 0.0;
        for (int c = 0; c < n; c += 32) {
            const int i = c + lane;
            const double th = i < n ? theta_at(i) : 0.0;
            if (i < n) {
                const double ph = 0.5 + 0.5 * tanh(th * pb.inv_delta);
                sum += hot ? ph : 1.0 - ph;
            }
            if (fz < 0.0) {
                const bool cross = i >= 1 && i < n && (hot ? th <= 0.0 : th >= 0.0);
                const unsigned m = __ballot_sync(kFull, cross);
                double before = __shfl_up_sync(kFull, th, 1);
                if (lane == 0) before = prev_last;
                if (m) {
                    const int first = __ffs(m) - 1;
                    const double a = __shfl_sync(kFull, before, first);
                    const double b = __shfl_sync(kFull, th, first);
                    fz = (double)(c + first - 1) + a / (a - b);
                }
            }
            prev_last = __shfl_sync(kFull, th, 31);
        }
        if (fz < 0.0) fz = (double)(n - 1);
        sum = warp_sum(sum);
        if (lane == 0) {
            out[line] = fz;
            out[nlines + line] = sum - 0.5;
        }
    }
}

cudaError_t launch_front(int precision, const Problem* dprob, const Problem& hp, int parity, int wall, double* out,
                         cudaStream_t s)
{
    const int nlines = wall <= 1 ? hp.ny : hp.nx;
    const int blocks = (nlines + 3) / 4;
    if (precision == 1) front_kernel<float><<<blocks, 128, 0, s>>>(dprob, parity, wall, out);
    else front_kernel<double><<<blocks, 128, 0, s>>>(dprob, parity, wall, out);
    return cudaGetLastError();
}

static int grid_for(long long n) { return (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16); }

cudaError_t launch_init_state(int precision, const Problem* dprob, const Problem& hp, const double* theta0,
                              int parity, DevStats* st, cudaStream_t s)
{
    const int g = grid_for((long long)hp.nx * hp.ny);
    // FP32 D2Q9 / D2Q5 states carry a shift (FP64 and D1Q3 tails stay zero)
    if (precision == 1 && hp.q != 3) {
        shift_kernel<<<1, 1024, 0, s>>>(dprob, theta0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
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
