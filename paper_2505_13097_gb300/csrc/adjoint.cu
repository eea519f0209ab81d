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
// D2Q9 (adj_march_kernel): with D_j(y) = dL/dq_j(y) including the wall
// corrections of node y, every output is lambda_j(x) = nu(x) + D_j(x + e_j),
// i.e. the forward pull with all directions reversed, and D_j(y), nu(y) depend
// on node y alone (its a, theta(t), theta(t+1)).  A warp owns a segment of
// 32*N columns and marches up tile_h rows, evaluating each row once and
// keeping, per lane, what the next output rows read:
//   D_2, D_5, D_6 of row y+1,  D_0, D_1, D_3 and nu of row y,  D_4, D_7, D_8 of row y-1.
// Shifts along x go through shuffles; the column on each side of the segment
// is evaluated by the warp together (lanes 0-8 and 16-24 hold the nine a of
// the left and right neighbour column, lanes 9-10 and 25-26 its two thetas).
// Directions that leave the lattice get nu alone; adj_links_kernel then adds
// the link-wise bounce-back terms at the boundary nodes that have them.
//
// FP32 form: a and lambda in FP32, interior nodes evaluated in FP32 with
// phi' = 2 e / (delta (1 + e)^2), e = exp(-2|theta|/delta), and
// phi(theta(t+1)) - phi(theta(t)) = sinh(x1 - x0) / (2 cosh x0 cosh x1),
// x = theta/delta, both free of cancellation; wall nodes in FP64.
// FP64 form: everything in FP64 with the formulas of the gather above.
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

// ---------------------------------------------------------------- D1Q3 gather
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
__global__ void __launch_bounds__(128) adj_step_kernel(const __grid_constant__ AdjArgs g)
{
    const Problem& pb = g.pb;
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

// ---------------------------------------------------------------- D2Q9 node terms
// Everything a D2Q9 node contributes to the reverse step, in FP64:
//   a (in)  -> D_j = dL/dq_j with the node's wall corrections (0 for unknown j),
//   link    -> (optional) link_j for outgoing j that leave the lattice,
//   nu, and the node's theta_D / Ste gradient terms.
struct NodeTerms {
    double nu, gw, gs;
    int wall;            // Dirichlet wall of the node, -1 if none
    unsigned link_mask;  // bit j: lambda_j(x) = nu + link_j
};

__device__ __noinline__ NodeTerms node_terms(const Problem& pb, double* a, double* link, double th0, double th1,
                                             int x, int y)
{
    NodeTerms r;
    double A = 0.0;
    for (int i = 8; i >= 0; --i) A += d2_w(i) * a[i];
    const double omc = 1.0 - pb.omega;
    unsigned unk = 0;
    for (int i = 1; i < 9; ++i) {
        const int sx = x - d2_ex(i), sy = y - d2_ey(i);
        if (sx < 0 || sx >= pb.nx || sy < 0 || sy >= pb.ny) unk |= 1u << i;
    }
    const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0);
    r.wall = -1;
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            r.wall = k;
            break;
        }
    r.gw = 0.0;
    r.gs = 0.0;
    r.link_mask = 0;
    if (r.wall >= 0) {
        const double td = pb.wall_theta[r.wall];
        const double mu = -omc * A;
        double wu = 0.0, B = 0.0;
        for (int i = 1; i < 9; ++i)
            if ((unk >> i) & 1) wu += d2_w(i);
        for (int i = 1; i < 9; ++i)
            if ((unk >> i) & 1) B += d2_w(i) * (omc * a[i] + mu);
        B /= wu;
        for (int j = 0; j < 9; ++j) a[j] = ((unk >> j) & 1) ? 0.0 : omc * a[j] + mu - B;
        r.nu = -B * dphi_of(th0, pb.inv_delta) * pb.inv_ste;
        r.gw = A + B * (1.0 + dphi_of(td, pb.inv_delta) * pb.inv_ste);
        r.gs = -B * (phi_of(td, pb.inv_delta) - phi_of(th0, pb.inv_delta)) * pb.inv_ste * pb.inv_ste;
        return r;
    }
    double mu;
    const double thr = pb.sat;
    if ((th0 >= thr && th1 >= thr) || (th0 <= -thr && th1 <= -thr)) {
        mu = pb.omega * A;   // F' = 1, phi'(theta) = 0
        r.nu = 0.0;
    } else {
        const double d1 = dphi_of(th1, pb.inv_delta), d0 = dphi_of(th0, pb.inv_delta);
        const double Fp = 1.0 + d1 * pb.inv_ste;
        mu = -omc * A + A / Fp;
        r.nu = A * d0 * pb.inv_ste / Fp;
        r.gs = A * (phi_of(th1, pb.inv_delta) - phi_of(th0, pb.inv_delta)) * pb.inv_ste * pb.inv_ste / Fp;
    }
    double dq[9];
    for (int j = 0; j < 9; ++j) dq[j] = omc * a[j] + mu;
    for (int j = 0; j < 9; ++j) a[j] = ((unk >> j) & 1) ? 0.0 : dq[j];
    for (int i = 1; i < 9; ++i)
        if ((unk >> i) & 1) {
            const int o = d2_opp(i);
            if (pb.bb_mode == 0 && !((unk >> o) & 1)) {
                a[o] += dq[i];
            } else {
                r.link_mask |= 1u << o;
                if (link) link[o] = dq[i];
            }
        }
    return r;
}

// ---------------------------------------------------------------- D2Q9 marching kernel
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS 4
#endif

template <typename P> struct AdjN;
template <> struct AdjN<float> { static constexpr int N = 2; };
template <> struct AdjN<double> { static constexpr int N = 1; };

__device__ __forceinline__ void ld_n(const float* p, float (&v)[2])
{
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ld_n(const double* p, double (&v)[1]) { v[0] = __ldg(p); }
__device__ __forceinline__ void ld_n(const double* p, double (&v)[2])
{
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void st_n(float* p, const float (&v)[2])
{
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
__device__ __forceinline__ void st_n(double* p, const double (&v)[1]) { *p = v[0]; }

// interior node (all nine q streamed, no Dirichlet value): mu, nu and the Ste term
__device__ __forceinline__ void interior_terms(float A, double th0, double th1, const AdjConst& c, float& mu,
                                               float& nu, float& gs)
{
    const float t0 = approx_float(th0), t1 = approx_float(th1);
    if ((t0 >= c.thr_f && t1 >= c.thr_f) || (t0 <= -c.thr_f && t1 <= -c.thr_f)) {
        mu = c.om_f * A;
        nu = 0.0f;
        return;
    }
    const float x0 = t0 * c.inv_delta_f, x1 = t1 * c.inv_delta_f;
    const float y0 = fabsf(x0), y1 = fabsf(x1);
    const float e0 = expf(-2.0f * y0), e1 = expf(-2.0f * y1);
    const float p0 = 1.0f + e0, p1 = 1.0f + e1;
    const float g0 = 2.0f * e0 / (p0 * p0) * c.inv_delta_f;   // phi'(theta(t))
    const float g1 = 2.0f * e1 / (p1 * p1) * c.inv_delta_f;   // phi'(theta(t+1))
    const float r = 1.0f / (1.0f + g1 * c.inv_ste_f);         // 1/F'
    mu = A * (r - c.omc_f);
    nu = A * g0 * c.inv_ste_f * r;
    const float d = (float)((th1 - th0) * c.inv_delta);
    const float dphi = fabsf(d) < 20.0f ? 2.0f * sinhf(d) * expf(-(y0 + y1)) / (p0 * p1)
                                        : 0.5f * (tanhf(x1) - tanhf(x0));
    gs += A * dphi * c.inv_ste2_f * r;
}
__device__ __forceinline__ void interior_terms(double A, double th0, double th1, const AdjConst& c, double& mu,
                                               double& nu, double& gs)
{
    if ((th0 >= c.thr && th1 >= c.thr) || (th0 <= -c.thr && th1 <= -c.thr)) {
        mu = c.om * A;
        nu = 0.0;
        return;
    }
    const double d1 = dphi_of(th1, c.inv_delta), d0 = dphi_of(th0, c.inv_delta);
    const double Fp = 1.0 + d1 * c.inv_ste;
    mu = -c.omc * A + A / Fp;
    nu = A * d0 * c.inv_ste / Fp;
    gs += A * (phi_of(th1, c.inv_delta) - phi_of(th0, c.inv_delta)) * c.inv_ste * c.inv_ste / Fp;
}

__device__ __forceinline__ float lat_w_f(int i) { return d2_wf(i); }
template <typename P> __device__ __forceinline__ P lat_w_p(int i);
template <> __device__ __forceinline__ float lat_w_p<float>(int i) { return lat_w_f(i); }
template <> __device__ __forceinline__ double lat_w_p<double>(int i) { return d2_w(i); }

// phi'(theta) and phi(theta_b) - phi(theta_a) in the population precision
// (FP32: from exp and sinh, free of cancellation; FP64: from tanh).
__device__ __forceinline__ float dphi_p(float, double th, const AdjConst& c)
{
    const float x = fabsf(approx_float(th) * c.inv_delta_f);
    const float e = expf(-2.0f * x);
    const float p = 1.0f + e;
    return 2.0f * e / (p * p) * c.inv_delta_f;
}
__device__ __forceinline__ double dphi_p(double, double th, const AdjConst& c) { return dphi_of(th, c.inv_delta); }
__device__ __forceinline__ float phidiff_p(float, double thb, double tha, const AdjConst& c)
{
    const float xa = approx_float(tha) * c.inv_delta_f, xb = approx_float(thb) * c.inv_delta_f;
    const float d = (float)((thb - tha) * c.inv_delta);
    if (fabsf(d) >= 20.0f) return 0.5f * (tanhf(xb) - tanhf(xa));
    const float ea = expf(-2.0f * fabsf(xa)), eb = expf(-2.0f * fabsf(xb));
    return 2.0f * sinhf(d) * expf(-(fabsf(xa) + fabsf(xb))) / ((1.0f + ea) * (1.0f + eb));
}
__device__ __forceinline__ double phidiff_p(double, double thb, double tha, const AdjConst& c)
{
    return phi_of(thb, c.inv_delta) - phi_of(tha, c.inv_delta);
}

// Per-lane sums of one launch: the interior Ste terms in the population
// precision (registers, converted once per tile); the wall-node terms (Ste,
// theta_D of each wall) in shared memory, touched only on wall rows and columns.
template <typename P>
struct AdjSums {
    P gs;
    double* wall;   // 5 doubles with stride blockDim.x: Ste, W, E, S, N
};

// Loads of one node row: the nine a, theta(t), theta(t+1), and this lane's
// element of the joint evaluation of the two columns beside the segment.
template <typename P, int N>
struct AdjLoads {
    P a[9][N];
    double t0[N], t1[N];
    P hv;
    double ht;
};

// D_j (into dq[.][k]) and nu of element k of a row: interior nodes with the
// interior terms, boundary nodes (bmask: bit 0..3 = on the W, E, S, N wall)
// with the wall closures of Sec. 4.2 transposed.  The link-wise bounce-back
// terms are left to adj_links_kernel.
template <typename P, int N>
__device__ __forceinline__ P node_row_terms(const Problem& pb, const AdjConst& c, const P (&a)[9][N], int k,
                                            double th0, double th1, unsigned bmask, bool count, P (&dq)[9][N],
                                            AdjSums<P>& sums)
{
    const P omc = sizeof(P) == 4 ? (P)c.omc_f : (P)c.omc;
    const P A = lat_w_p<P>(0) * a[0][k] + lat_w_p<P>(1) * ((a[1][k] + a[2][k]) + (a[3][k] + a[4][k])) +
                lat_w_p<P>(5) * ((a[5][k] + a[6][k]) + (a[7][k] + a[8][k]));
    if (bmask == 0) {
        P mu, nu, gs = 0;
        interior_terms(A, th0, th1, c, mu, nu, gs);
        if (count) sums.gs += gs;
#pragma unroll
        for (int i = 0; i < 9; ++i) dq[i][k] = omc * a[i][k] + mu;
        return nu;
    }
    // q_i not defined by streaming: sources beyond the W, E, S, N walls
    const unsigned unk = ((bmask & 1u) ? 0x122u : 0u) | ((bmask & 2u) ? 0x0c8u : 0u) | ((bmask & 4u) ? 0x064u : 0u) |
                         ((bmask & 8u) ? 0x190u : 0u);
    int wall = -1;
    for (int w = 3; w >= 0; --w)
        if (((bmask >> w) & 1u) && pb.wall_kind[w] == 1) wall = w;
    if (wall >= 0) {
        const P mu = -omc * A;
        P wu = 0, B = 0;
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((unk >> i) & 1u) {
                wu += lat_w_p<P>(i);
                B += lat_w_p<P>(i) * (omc * a[i][k] + mu);
            }
        B /= wu;
#pragma unroll
        for (int j = 0; j < 9; ++j) dq[j][k] = ((unk >> j) & 1u) ? (P)0 : omc * a[j][k] + mu - B;
        const double td = pb.wall_theta[wall];
        const P inv_ste = sizeof(P) == 4 ? (P)c.inv_ste_f : (P)c.inv_ste;
        if (count) {
            sums.wall[(1 + wall) * kWarpsPerBlock * 32] += (double)(A + B * (1 + dphi_p(P(0), td, c) * inv_ste));
            sums.wall[0] += (double)(-B * phidiff_p(P(0), td, th0, c) * inv_ste * inv_ste);
        }
        return -B * dphi_p(P(0), th0, c) * inv_ste;
    }
    P mu, nu, gs = 0;
    interior_terms(A, th0, th1, c, mu, nu, gs);
    if (count) sums.gs += gs;
    P d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = omc * a[i][k] + mu;
#pragma unroll
    for (int j = 0; j < 9; ++j) dq[j][k] = ((unk >> j) & 1u) ? (P)0 : d[j];
    if (pb.bb_mode == 0) {
        // mirror bounce-back: q_i = Omega_o pulled along e_o, o = opp(i), when that one is known
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const int o = d2_opp(i);
            if (((unk >> i) & 1u) && !((unk >> o) & 1u)) dq[o][k] += d[i];
        }
    }
    return nu;
}

template <typename P>
__device__ __forceinline__ void adj_tile(const Problem& pb, const AdjArgs& g, const P* __restrict__ ain,
                                         P* __restrict__ aout, int seg, int ya, int yb, const AdjConst& c,
                                         AdjSums<P>& sums)
{
    constexpr int N = AdjN<P>::N;
    constexpr int W = 32 * N;
    const int lane = threadIdx.x & 31;
    const int segx = seg * W;
    const int x0 = segx + lane * N;
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    const int nx = pb.nx, ny = pb.ny;
    const bool has_left = segx > 0;
    const bool has_right = segx + W < nx;
    const int hl = lane & 15;
    const int hx = lane < 16 ? segx - 1 : segx + W;
    const bool hside = lane < 16 ? has_left : has_right;
    const double* __restrict__ th0p = g.theta_t;
    const double* __restrict__ th1p = g.theta_t1;
    const P omc = sizeof(P) == 4 ? (P)c.omc_f : (P)c.omc;

    auto issue = [&](AdjLoads<P, N>& L, int r) {
        if (r < 0 || r >= ny) return;
        const long long ro = (long long)(r + 1) * pitch;
#pragma unroll
        for (int i = 0; i < 9; ++i) ld_n(static_cast<const P*>(g.in_plane[i]) + ro + x0, L.a[i]);
        ld_n(th0p + (long long)r * pitch + x0, L.t0);
        ld_n(th1p + (long long)r * pitch + x0, L.t1);
        L.hv = (hside && hl < 9) ? __ldg(ain + hl * pl + ro + hx) : (P)0;
        L.ht = (hside && hl == 9) ? __ldg(th0p + (long long)r * pitch + hx)
                                  : ((hside && hl == 10) ? __ldg(th1p + (long long)r * pitch + hx) : 0.0);
    };

    AdjLoads<P, N> L, Ln;
    P k4[N], k7[N], k8[N], knu[N];   // D_4, D_7, D_8 (shifted) and nu of the row below
    issue(L, ya - 1);
    for (int r = ya - 1; r <= yb; ++r) {
        if (r + 1 <= yb) issue(Ln, r + 1);
        P dq[9][N], nu[N];
        P hL3 = 0, hL6 = 0, hL7 = 0, hR1 = 0, hR5 = 0, hR8 = 0;
        if (r < 0 || r >= ny) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                nu[k] = (P)0;
#pragma unroll
                for (int i = 0; i < 9; ++i) dq[i][k] = (P)0;
            }
        } else {
            const bool count = r >= ya && r < yb;
            const bool wall_row = r == 0 || r == ny - 1;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int x = x0 + k;
                const unsigned bmask = (x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u) | (r == 0 ? 4u : 0u) |
                                       (r == ny - 1 ? 8u : 0u);
                if (x >= nx) {
                    nu[k] = (P)0;
#pragma unroll
                    for (int i = 0; i < 9; ++i) dq[i][k] = (P)0;
                } else {
                    nu[k] = node_row_terms<P, N>(pb, c, L.a, k, L.t0[k], L.t1[k], bmask, count, dq, sums);
                }
            }
            // the columns beside the segment, evaluated by the warp together:
            // lanes 0-15 the left one, lanes 16-31 the right one
            P Ah = hl < 9 ? lat_w_p<P>(hl) * L.hv : (P)0;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) Ah += __shfl_xor_sync(kFull, Ah, o);
            const double t0h = __shfl_sync(kFull, L.ht, (lane & 16) | 9);
            const double t1h = __shfl_sync(kFull, L.ht, (lane & 16) | 10);
            P muh, nuh, gsh = 0;
            interior_terms(Ah, t0h, t1h, c, muh, nuh, gsh);
            const P dqh = omc * L.hv + muh;
            // lane 0 takes D_3, D_6, D_7 of the left column, lane 31 D_1, D_5, D_8 of the right one
            const P v1 = __shfl_sync(kFull, dqh, lane < 16 ? 3 : 17);
            const P v2 = __shfl_sync(kFull, dqh, lane < 16 ? 6 : 21);
            const P v3 = __shfl_sync(kFull, dqh, lane < 16 ? 7 : 24);
            if (hside) {
                hL3 = v1; hL6 = v2; hL7 = v3;
                hR1 = v1; hR5 = v2; hR8 = v3;
            }
            // a neighbour column on a wall row or on the east wall: its own wall terms
            if ((lane == 0 && has_left && wall_row) || (lane == 31 && has_right && (wall_row || hx == nx - 1))) {
                const long long ro = (long long)(r + 1) * pitch + hx;
                P ah[9][N], dh[9][N];
                for (int i = 0; i < 9; ++i) ah[i][0] = ain[i * pl + ro];
                const unsigned bmask = (hx == nx - 1 ? 2u : 0u) | (r == 0 ? 4u : 0u) | (r == ny - 1 ? 8u : 0u);
                node_row_terms<P, N>(pb, c, ah, 0, th0p[(long long)r * pitch + hx], th1p[(long long)r * pitch + hx],
                                     bmask, false, dh, sums);
                hL3 = dh[3][0]; hL6 = dh[6][0]; hL7 = dh[7][0];
                hR1 = dh[1][0]; hR5 = dh[5][0]; hR8 = dh[8][0];
            }
        }
        P d1[N], d3[N], d5[N], d6[N], d7[N], d8[N];
        from_right<P, N>(dq[1], hR1, lane, d1);   // output x reads D_1(x + 1)
        from_left<P, N>(dq[3], hL3, lane, d3);    // D_3(x - 1)
        from_right<P, N>(dq[5], hR5, lane, d5);   // D_5(x + 1), read by the row below
        from_left<P, N>(dq[6], hL6, lane, d6);    // D_6(x - 1), read by the row below
        from_left<P, N>(dq[7], hL7, lane, d7);    // D_7(x - 1), read by the row above
        from_right<P, N>(dq[8], hR8, lane, d8);   // D_8(x + 1), read by the row above
        P o[N];
        if (r >= ya && r < yb) {
            // this row: lambda_j = nu + D_j(x + e_j) for e_y(j) = 0 and -1
            const long long ro = (long long)(r + 1) * pitch + x0;
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = nu[k] + dq[0][k];
            st_n(static_cast<P*>(g.out_plane[0]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = nu[k] + d1[k];
            st_n(static_cast<P*>(g.out_plane[1]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = nu[k] + d3[k];
            st_n(static_cast<P*>(g.out_plane[3]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = nu[k] + k4[k];
            st_n(static_cast<P*>(g.out_plane[4]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = nu[k] + k7[k];
            st_n(static_cast<P*>(g.out_plane[7]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = nu[k] + k8[k];
            st_n(static_cast<P*>(g.out_plane[8]) + ro, o);
        }
        if (r - 1 >= ya) {
            // the row below: lambda_j for e_y(j) = +1
            const long long ro = (long long)r * pitch + x0;
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = knu[k] + dq[2][k];
            st_n(static_cast<P*>(g.out_plane[2]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = knu[k] + d5[k];
            st_n(static_cast<P*>(g.out_plane[5]) + ro, o);
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = knu[k] + d6[k];
            st_n(static_cast<P*>(g.out_plane[6]) + ro, o);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            k4[k] = dq[4][k]; k7[k] = d7[k]; k8[k] = d8[k]; knu[k] = nu[k];
        }
        L = Ln;
    }
}

template <typename P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, LBM_ADJ_MIN_BLOCKS) adj_march_kernel(const __grid_constant__ AdjArgs g)
{
    __shared__ double wall_sums[5 * kWarpsPerBlock * 32];
    const Problem& pb = g.pb;
    const P* ain = static_cast<const P*>(g.adj_in);
    P* aout = static_cast<P*>(g.adj_out);
    AdjSums<P> sums;
    sums.gs = 0;
    sums.wall = wall_sums + threadIdx.x;
    for (int k = 0; k < 5; ++k) sums.wall[k * kWarpsPerBlock * 32] = 0.0;
    double gs_total = 0.0;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = warp; t < g.ntiles; t += nwarps) {
        const int seg = t % pb.nseg;
        const int ya = (t / pb.nseg) * g.tile_h;
        const int yb = min(pb.ny, ya + g.tile_h);
        adj_tile<P>(pb, g, ain, aout, seg, ya, yb, g.c, sums);
        gs_total += (double)sums.gs;   // one conversion per tile
        sums.gs = 0;
    }
    gs_total += sums.wall[0];
    DevStats* st = g.stats;
    for (int w = 0; w < 4; ++w) {
        if (pb.wall_kind[w] != 1) continue;
        const double v = warp_sum(sums.wall[(1 + w) * kWarpsPerBlock * 32]);
        if ((threadIdx.x & 31) == 0 && v != 0.0) acc_add(&st->g_wall[w], v);
    }
    gs_total = warp_sum(gs_total);
    if ((threadIdx.x & 31) == 0 && gs_total != 0.0) acc_add(&st->g_ste, gs_total);
}

// Link-wise bounce-back terms (Sec. 4.2): at a boundary node whose q_i is
// copied from its own Omega_o, o = opp(i), lambda_o = nu + dL/dq_i.  One
// thread per boundary node (corners_only: the four corners, the only nodes
// with such terms under mirror bounce-back); runs after adj_march_kernel,
// which wrote nu there.
template <typename P>
__global__ void adj_links_kernel(const __grid_constant__ AdjArgs g, int corners_only)
{
    const Problem& pb = g.pb;
    const int nx = pb.nx, ny = pb.ny;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int x, y;
    if (corners_only) {
        if (k >= 4) return;
        x = (k & 1) ? nx - 1 : 0;
        y = (k & 2) ? ny - 1 : 0;
    } else if (k < nx) {
        x = k; y = 0;
    } else if (k < 2 * nx) {
        x = k - nx; y = ny - 1;
    } else if (k < 2 * nx + (ny - 2)) {
        x = 0; y = k - 2 * nx + 1;
    } else if (k < 2 * nx + 2 * (ny - 2)) {
        x = nx - 1; y = k - 2 * nx - (ny - 2) + 1;
    } else {
        return;
    }
    // nodes without such terms leave at once: Dirichlet nodes, and under mirror
    // bounce-back every node whose unknown directions all have a known opposite
    const unsigned bmask = (x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u) | (y == 0 ? 4u : 0u) | (y == ny - 1 ? 8u : 0u);
    for (int w = 0; w < 4; ++w)
        if (((bmask >> w) & 1u) && pb.wall_kind[w] == 1) return;
    const unsigned unk = ((bmask & 1u) ? 0x122u : 0u) | ((bmask & 2u) ? 0x0c8u : 0u) | ((bmask & 4u) ? 0x064u : 0u) |
                         ((bmask & 8u) ? 0x190u : 0u);
    bool any = false;
    for (int i = 1; i < 9; ++i)
        if (((unk >> i) & 1u) && (pb.bb_mode == 1 || ((unk >> d2_opp(i)) & 1u))) any = true;
    if (!any) return;
    const P* ain = static_cast<const P*>(g.adj_in);
    P* aout = static_cast<P*>(g.adj_out);
    const long long ro = (long long)(y + 1) * pb.pitch + x;
    double a[9], link[9];
    for (int i = 0; i < 9; ++i) {
        a[i] = (double)ain[i * pb.plane + ro];
        link[i] = 0.0;
    }
    const NodeTerms t = node_terms(pb, a, link, g.theta_t[(long long)y * pb.pitch + x],
                                   g.theta_t1[(long long)y * pb.pitch + x], x, y);
    for (int j = 1; j < 9; ++j)
        if ((t.link_mask >> j) & 1) aout[j * pb.plane + ro] = (P)(t.nu + link[j]);
}

// ---------------------------------------------------------------- seed and finish
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
    if (hp.q == 9) {
        const int blocks = (a.ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
        if (precision == 1) adj_march_kernel<float><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
        else adj_march_kernel<double><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
        // link-wise terms: every boundary node that is not Dirichlet under
        // link-wise bounce-back, the corners that are not under mirror bounce-back
        const int corners_only = hp.bb_mode == 0;
        bool needed = !corners_only;
        if (corners_only)
            for (int k = 0; k < 4; ++k) {
                const int wx = (k & 1) ? 1 : 0, wy = (k & 2) ? 3 : 2;   // the corner's two walls
                if (hp.wall_kind[wx] != 1 && hp.wall_kind[wy] != 1) needed = true;
            }
        if (needed) {
            const int nb = corners_only ? 4 : 2 * hp.nx + 2 * (hp.ny - 2);
            if (precision == 1) adj_links_kernel<float><<<(nb + 127) / 128, 128, 0, s>>>(a, corners_only);
            else adj_links_kernel<double><<<(nb + 127) / 128, 128, 0, s>>>(a, corners_only);
        }
        return cudaGetLastError();
    }
    const int g = agrid((long long)hp.nx * hp.ny);
    if (precision == 1) adj_step_kernel<3, float><<<g, 128, 0, s>>>(a);
    else adj_step_kernel<3, double><<<g, 128, 0, s>>>(a);
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
