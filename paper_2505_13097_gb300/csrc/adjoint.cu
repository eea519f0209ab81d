// Discrete adjoint of the IREBM step (D2Q9 and D1Q3).
//
// Forward step per node y, in the stored-Omega form of the kernels:
//   theta(y) = sum_i Omega_i(y),  q_i(y) = Omega_i(y - e_i) or the wall closure,
//   m0(y) = sum_i q_i(y),  theta'(y) = root of Eq. (14) (theta_D on Dirichlet nodes),
//   Omega~_i(y) = (1-omega) q_i(y) + w_i (theta'(y) - (1-omega) m0(y)).
// With a_i(y) = dL/dOmega~_i(y) and A = sum_i w_i a_i, the transpose is
//   dL/dq_i(y) = (1-omega) a_i(y) + mu(y),
//   mu(y)  = -(1-omega) A + A/F'          (Newton node; implicit function theorem,
//            F' = 1 + phi'(theta')/Ste)
//   mu(y)  = -(1-omega) A                 (Dirichlet node: theta' = theta_D)
//   nu(y)  = dL/dtheta(y) = A phi'(theta)/(Ste F')   (Dirichlet: -B phi'(theta)/Ste)
// and the gradient of the old populations gathers along the streaming links:
//   lambda_j(x) = nu(x) + dL/dq_j(x + e_j) [+ wall corrections]   if x + e_j is inside,
//   lambda_j(x) = nu(x) + link_j(x)                               otherwise.
// Wall corrections transpose Sec. 4.2: mirror bounce-back sends dL/dq_i to the
// known opposite q, link-wise bounce-back to Omega at the node, the Dirichlet
// closure to the known q (-B), to theta_D and to theta.  Ste and theta_D
// gradients accumulate in fixed point (order independent).
//
// This version evaluates, for every node, the scalars of its q neighbours
// again (9 node evaluations per node for D2Q9).
#include "lbm_device.cuh"

namespace lbm {

template <int Q> __device__ __forceinline__ int lex(int i) { return Q == 9 ? d2_ex(i) : d1_ex(i); }
template <int Q> __device__ __forceinline__ int ley(int i) { return Q == 9 ? d2_ey(i) : 0; }
template <int Q> __device__ __forceinline__ double lw(int i) { return Q == 9 ? d2_w(i) : d1_w(i); }
template <int Q> __device__ __forceinline__ int lopp(int i) { return Q == 9 ? d2_opp(i) : (i == 0 ? 0 : 3 - i); }

__device__ __forceinline__ double dphi_of(double x, double inv_delta)
{
    const double t = tanh(x * inv_delta);
    return 0.5 * (1.0 - t) * (1.0 + t) * inv_delta;
}

template <int Q>
struct NodeAdj {
    double mu, nu;
    double corr[Q];   // added to dL/dq_j(y) for the neighbour y - e_j
    double link[Q];   // lambda_j(y) for outgoing j (y + e_j outside)
    double gwall, gste;
    int wall;         // Dirichlet wall index of this node, -1 if none
};

template <int Q, typename P>
__device__ NodeAdj<Q> node_adj(const Problem& pb, const P* __restrict__ ain, const double* __restrict__ th0p,
                               const double* __restrict__ th1p, int x, int y)
{
    NodeAdj<Q> r;
    double a[Q];
    const long long off = (long long)(y + 1) * pb.pitch + x;
    for (int i = 0; i < Q; ++i) {
        a[i] = (double)ain[i * pb.plane + off];
        r.corr[i] = 0.0;
        r.link[i] = 0.0;
    }
    const double th0 = th0p[(long long)y * pb.pitch + x];
    const double th1 = th1p[(long long)y * pb.pitch + x];
    double A = 0.0;
    for (int i = Q - 1; i >= 0; --i) A += lw<Q>(i) * a[i];
    const double omc = 1.0 - pb.omega;
    unsigned unk = 0;
    for (int i = 1; i < Q; ++i) {
        const int sx = x - lex<Q>(i), sy = y - ley<Q>(i);
        if (sx < 0 || sx >= pb.nx || sy < 0 || sy >= pb.ny) unk |= 1u << i;
    }
    const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) |
                      (Q == 9 ? ((y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0)) : 0);
    r.wall = -1;
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            r.wall = k;
            break;
        }
    r.gwall = 0.0;
    r.gste = 0.0;
    if (r.wall >= 0) {
        const double td = pb.wall_theta[r.wall];
        r.mu = -omc * A;
        double wu = 0.0, B = 0.0;
        for (int i = 1; i < Q; ++i)
            if ((unk >> i) & 1) wu += lw<Q>(i);
        for (int i = 1; i < Q; ++i)
            if ((unk >> i) & 1) B += lw<Q>(i) * (omc * a[i] + r.mu);
        B /= wu;
        for (int j = 0; j < Q; ++j)
            if (!((unk >> j) & 1)) r.corr[j] = -B;
        r.nu = -B * dphi_of(th0, pb.inv_delta) * pb.inv_ste;
        r.gwall = A + B * (1.0 + dphi_of(td, pb.inv_delta) * pb.inv_ste);
        r.gste = -B * (phi_of(td, pb.inv_delta) - phi_of(th0, pb.inv_delta)) * pb.inv_ste * pb.inv_ste;
    } else {
        const double thr = kSat * pb.delta;
        const bool sat = (th0 >= thr && th1 >= thr) || (th0 <= -thr && th1 <= -thr);
        if (sat) {
            r.mu = pb.omega * A;   // F' = 1, phi'(theta) = 0
            r.nu = 0.0;
        } else {
            const double d1 = dphi_of(th1, pb.inv_delta), d0 = dphi_of(th0, pb.inv_delta);
            const double Fp = 1.0 + d1 * pb.inv_ste;
            r.mu = -omc * A + A / Fp;
            r.nu = A * d0 * pb.inv_ste / Fp;
            r.gste = A * (phi_of(th1, pb.inv_delta) - phi_of(th0, pb.inv_delta)) * pb.inv_ste * pb.inv_ste / Fp;
        }
        for (int i = 1; i < Q; ++i)
            if ((unk >> i) & 1) {
                const int o = lopp<Q>(i);
                const double dq = omc * a[i] + r.mu;
                if (pb.bb_mode == 0 && !((unk >> o) & 1)) r.corr[o] += dq;
                else r.link[o] += dq;
            }
    }
    return r;
}

template <int Q, typename P>
__global__ void __launch_bounds__(128) adj_step_kernel(AdjArgs g)
{
    const Problem& pb = *g.prob;
    DevStats* st = g.stats;
    const P* ain = static_cast<const P*>(g.adj_in);
    P* aout = static_cast<P*>(g.adj_out);
    const long long n = (long long)pb.nx * pb.ny;
    double gw[4] = {0, 0, 0, 0}, gs = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        NodeAdj<Q> self = node_adj<Q, P>(pb, ain, g.theta_t, g.theta_t1, x, y);
        if (self.wall >= 0) gw[self.wall] += self.gwall;
        gs += self.gste;
        const long long off = (long long)(y + 1) * pb.pitch + x;
        for (int j = 0; j < Q; ++j) {
            const int xx = x + lex<Q>(j), yy = y + ley<Q>(j);
            double lam = self.nu;
            if (xx >= 0 && xx < pb.nx && yy >= 0 && yy < pb.ny) {
                if (j == 0) {
                    lam += (1.0 - pb.omega) * (double)ain[off] + self.mu + self.corr[0];
                } else {
                    NodeAdj<Q> nb = node_adj<Q, P>(pb, ain, g.theta_t, g.theta_t1, xx, yy);
                    lam += (1.0 - pb.omega) * (double)ain[j * pb.plane + (long long)(yy + 1) * pb.pitch + xx] + nb.mu +
                           nb.corr[j];
                }
            } else {
                lam += self.link[j];
            }
            aout[j * pb.plane + off] = (P)lam;
        }
    }
    for (int w = 0; w < 4; ++w) {
        const double v = warp_sum(gw[w]);
        if ((threadIdx.x & 31) == 0) acc_add(&st->g_wall[w], v);
    }
    gs = warp_sum(gs);
    if ((threadIdx.x & 31) == 0) acc_add(&st->g_ste, gs);
}

template <int Q, typename P>
__global__ void adj_seed_kernel(const Problem* dprob, const double* __restrict__ thT, const double* __restrict__ target,
                                void* adj, DevStats* st)
{
    const Problem& pb = *dprob;
    P* a = static_cast<P*>(adj);
    const long long n = (long long)pb.nx * pb.ny;
    double L = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        const double th = thT[(long long)y * pb.pitch + x];
        const double d = phi_of(th, pb.inv_delta) - target[k];
        L += 0.5 * d * d;
        const double s = d * dphi_of(th, pb.inv_delta);   // dL/dtheta_T; theta_T = sum_i Omega_i
        for (int i = 0; i < Q; ++i) a[i * pb.plane + (long long)(y + 1) * pb.pitch + x] = (P)s;
    }
    L = warp_sum(L);
    if ((threadIdx.x & 31) == 0) acc_add(&st->loss, L);
}

template <int Q, typename P>
__global__ void adj_finish_kernel(const Problem* dprob, const void* adj0, double* g_theta0, DevStats* st)
{
    const Problem& pb = *dprob;
    const P* a = static_cast<const P*>(adj0);
    const long long n = (long long)pb.nx * pb.ny;
    double gw[4] = {0, 0, 0, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % pb.nx), y = (int)(k / pb.nx);
        double s = 0.0;
        for (int i = Q - 1; i >= 0; --i) s += lw<Q>(i) * (double)a[i * pb.plane + (long long)(y + 1) * pb.pitch + x];
        // Omega_i(0) = w_i theta0, or w_i theta_D on a Dirichlet node
        const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) |
                          (Q == 9 ? ((y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0)) : 0);
        int wall = -1;
        for (int w = 0; w < 4; ++w)
            if (((walls >> w) & 1) && pb.wall_kind[w] == 1) {
                wall = w;
                break;
            }
        if (wall >= 0) {
            gw[wall] += s;
            g_theta0[k] = 0.0;
        } else {
            g_theta0[k] = s;
        }
    }
    for (int w = 0; w < 4; ++w) {
        const double v = warp_sum(gw[w]);
        if ((threadIdx.x & 31) == 0) acc_add(&st->g_wall[w], v);
    }
}

static int agrid(long long n) { return (int)((n + 127) / 128 < 152 * 32 ? (n + 127) / 128 : 152 * 32); }

cudaError_t launch_adj_seed(int precision, const Problem* dprob, const Problem& hp, const double* theta_T,
                            const double* phi_target, void* adj, DevStats* st, cudaStream_t s)
{
    const int g = agrid((long long)hp.nx * hp.ny);
    if (hp.q == 9) {
        if (precision == 1) adj_seed_kernel<9, float><<<g, 128, 0, s>>>(dprob, theta_T, phi_target, adj, st);
        else adj_seed_kernel<9, double><<<g, 128, 0, s>>>(dprob, theta_T, phi_target, adj, st);
    } else {
        if (precision == 1) adj_seed_kernel<3, float><<<g, 128, 0, s>>>(dprob, theta_T, phi_target, adj, st);
        else adj_seed_kernel<3, double><<<g, 128, 0, s>>>(dprob, theta_T, phi_target, adj, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_step(int precision, const AdjArgs& a, const Problem& hp, cudaStream_t s)
{
    const int g = agrid((long long)hp.nx * hp.ny);
    if (hp.q == 9) {
        if (precision == 1) adj_step_kernel<9, float><<<g, 128, 0, s>>>(a);
        else adj_step_kernel<9, double><<<g, 128, 0, s>>>(a);
    } else {
        if (precision == 1) adj_step_kernel<3, float><<<g, 128, 0, s>>>(a);
        else adj_step_kernel<3, double><<<g, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(int precision, const Problem* dprob, const Problem& hp, const void* adj0,
                              double* g_theta0, DevStats* st, cudaStream_t s)
{
    const int g = agrid((long long)hp.nx * hp.ny);
    if (hp.q == 9) {
        if (precision == 1) adj_finish_kernel<9, float><<<g, 128, 0, s>>>(dprob, adj0, g_theta0, st);
        else adj_finish_kernel<9, double><<<g, 128, 0, s>>>(dprob, adj0, g_theta0, st);
    } else {
        if (precision == 1) adj_finish_kernel<3, float><<<g, 128, 0, s>>>(dprob, adj0, g_theta0, st);
        else adj_finish_kernel<3, double><<<g, 128, 0, s>>>(dprob, adj0, g_theta0, st);
    }
    return cudaGetLastError();
}

}  // namespace lbm
