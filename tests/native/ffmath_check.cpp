// Host check of the float-float helpers the FP32 form's Newton solves use
// (paper_2505_13097_gb300/csrc/ffmath.cuh, compiled here for the CPU with
// plain IEEE float operations): exp(y) for y <= 0 and phi(x) = 1/(1 + exp(-2x/delta))
// (Sec. 4.1) with 1 - phi, against long double on seeded random inputs.
// Prints the largest errors; the Python test holds them to their bounds.
#include "../../paper_2505_13097_gb300/csrc/ffmath.cuh"

#include <cmath>
#include <cstdio>
#include <random>

using lbm::ff;

static long double ld(const ff& a) { return (long double)a.hi + (long double)a.lo; }
static ff split(double v)
{
    const float h = (float)v;
    return lbm::two_sum(h, (float)(v - (double)h));
}

int main()
{
    std::mt19937_64 g(20250513);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    long double exp_rel = 0, phi_abs = 0, phic_rel = 0, quot_rel = 0, prod_rel = 0;
    for (int i = 0; i < 400000; ++i) {
        // exp on [-40, 0], denser near 0
        const double yd = -40.0 * U(g) * U(g);
        const ff y = split(yd);
        const long double ex = expl(ld(y));
        exp_rel = fmaxl(exp_rel, fabsl(ld(lbm::ff_exp_nonpos(y)) - ex) / ex);
        // phi over the band and beyond: x in [-0.2, 0.2], 1/delta in [67, 200]
        const ff x = split((U(g) - 0.5) * 0.4);
        const ff id = split(100.0 / (0.5 + U(g)));
        const lbm::PhiFF p = lbm::ff_phi(x, id);
        const long double z = ld(x) * ld(id);
        const long double ph = 1.0L / (1.0L + expl(-2.0L * z)), phc = 1.0L / (1.0L + expl(2.0L * z));
        phi_abs = fmaxl(phi_abs, fabsl(ld(p.phi) - ph));
        if (phc > 1e-12L) phic_rel = fmaxl(phic_rel, fabsl(ld(p.phic) - phc) / phc);
        // quotient and product of float-float values
        const ff a = split((U(g) - 0.5) * 1e3), b = split(0.5 + U(g));
        quot_rel = fmaxl(quot_rel, fabsl(ld(lbm::ff_quot(a, b)) - ld(a) / ld(b)) / fabsl(ld(a) / ld(b)));
        prod_rel = fmaxl(prod_rel, fabsl(ld(lbm::ff_prod(a, b)) - ld(a) * ld(b)) / fabsl(ld(a) * ld(b)));
    }
    std::printf("exp_rel %.6Le\nphi_abs %.6Le\nphic_rel %.6Le\nquot_rel %.6Le\nprod_rel %.6Le\n", exp_rel, phi_abs,
                phic_rel, quot_rel, prod_rel);
    return 0;
}
