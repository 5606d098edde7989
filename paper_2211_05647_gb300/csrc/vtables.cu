// vtables.cu -- host-side velocity-grid tables of the kinetic update
// (Sec. 5.2, Eq. 20-24): node velocity, current weight w, F0 and its v_par
// derivative, volume element, and the collision law's s(v)|v| with its
// F0-weighted mean.  Shared by the solver and the batched driver.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace fp {

namespace {

// Druyvesteyn F0 of unit density, A exp(-(eps/eps0)^2) with eps = m v^2 / 2;
// eps0 makes the mean energy 3/2 e Te (mean energy = eps0 Gamma(5/4)/Gamma(3/4)),
// A makes the velocity-space integral 1.
struct Druyvesteyn {
    double eps0, A;
    explicit Druyvesteyn(double te_ev)
        : eps0(1.5 * kQe * te_ev * std::tgamma(0.75) / std::tgamma(1.25)),
          A(1.0 / (kPi * std::tgamma(0.75) * std::pow(2.0 * eps0 / kMe, 1.5)))
    {
    }
    double f(double v2) const   // F0 at |v|^2 = v2
    {
        const double x = 0.5 * kMe * v2 / eps0;
        return A * std::exp(-x * x);
    }
    // 1-D marginal over the two other components and its derivative
    double marg1(double u) const
    {
        return 0.5 * std::pow(kPi, 1.5) * A * (2.0 * eps0 / kMe) * std::erfc(0.5 * kMe * u * u / eps0);
    }
    double marg1_du(double u) const { return -2.0 * kPi * u * f(u * u); }
    // 2-D marginal over the third component t and its u derivative,
    // dh/du = -(2 m u / eps0^2) int eps F0 dt.  Trapezoid rule in t on
    // [-6, 6] sqrt(2 eps0/m) (the integrand is smooth and falls below 1e-300
    // of its peak there, so the rule converges faster than any power of the
    // step); 256 points per unit of sqrt(2 eps0/m).
    void marg2(double u, double w, double *h, double *dh) const
    {
        const double unit = std::sqrt(2.0 * eps0 / kMe), step = unit / 256.0;
        const int n = 6 * 256;
        double s0 = 0.0, s1 = 0.0;
        for (int q = -n; q <= n; ++q) {
            const double t = q * step, v2 = u * u + w * w + t * t;
            const double c = (q == -n || q == n) ? 0.5 : 1.0;
            const double fv = f(v2);
            s0 += c * fv;
            s1 += c * 0.5 * kMe * v2 * fv;
        }
        *h = s0 * step;
        *dh = -(2.0 * kMe * u / (eps0 * eps0)) * s1 * step;
    }
};

double table_sigma(const fdtd_plasma_desc &p, double v)
{
    const int64_t n = p.s_n;
    if (v <= p.s_speed[0]) return p.s_sigma[0];
    if (v >= p.s_speed[n - 1]) return p.s_sigma[n - 1];
    const int64_t k = std::upper_bound(p.s_speed, p.s_speed + n, v) - p.s_speed - 1;
    const double r = (v - p.s_speed[k]) / (p.s_speed[k + 1] - p.s_speed[k]);
    return p.s_sigma[k] + r * (p.s_sigma[k + 1] - p.s_sigma[k]);
}

}  // namespace

const char *check_velocity_model(const fdtd_plasma_desc &p)
{
    if (p.f0_model != FDTD_F0_MAXWELL && p.f0_model != FDTD_F0_DRUYVESTEYN) return "bad f0_model";
    if (p.nu_model != FDTD_NU_NSV && p.nu_model != FDTD_NU_CONST && p.nu_model != FDTD_NU_TABLE)
        return "bad nu_model";
    if (p.nu_model == FDTD_NU_TABLE) {
        if (!p.s_speed || !p.s_sigma || p.s_n < 2) return "nu_model TABLE needs s_speed, s_sigma and s_n >= 2";
        for (int64_t k = 0; k < p.s_n; ++k) {
            if (!std::isfinite(p.s_speed[k]) || !(p.s_speed[k] >= 0) || !std::isfinite(p.s_sigma[k]) ||
                !(p.s_sigma[k] >= 0))
                return "s table entries must be finite, speeds and cross-sections >= 0";
            if (k && !(p.s_speed[k] > p.s_speed[k - 1])) return "s table speeds must be strictly ascending";
        }
    }
    return nullptr;
}

bool velocity_tables(const fdtd_plasma_desc &p, VTab &t)
{
    const double vth = std::sqrt(kQe * p.te_ev / kMe);
    const double vmax = p.vmax_vth * vth;
    const double two_vth2 = 2.0 * vth * vth;
    const bool dru = p.f0_model == FDTD_F0_DRUYVESTEYN;
    const Druyvesteyn D(p.te_ev);
    if (p.vgrid == FDTD_VGRID_SIGNED1D) {
        const double dv = 2.0 * vmax / p.nv;
        for (int a = 0; a < p.nv; ++a) {
            const double va = ((double)a + 0.5 - 0.5 * p.nv) * dv;
            if (dru) {
                t.f0.push_back(D.marg1(va));
                t.f0p.push_back(D.marg1_du(va));
            } else {
                const double g = std::exp(-va * va / two_vth2) / std::sqrt(kPi * two_vth2);
                t.f0.push_back(g);
                t.f0p.push_back(-va / (vth * vth) * g);
            }
            t.v.push_back(va); t.w.push_back(va * dv); t.dV.push_back(dv); t.speed.push_back(std::fabs(va));
        }
    } else if (p.vgrid == FDTD_VGRID_CART2D) {
        const double dvp = 2.0 * vmax / p.nv, dvq = 2.0 * vmax / p.nv_perp;
        for (int a = 0; a < p.nv; ++a) {
            const double va = ((double)a + 0.5 - 0.5 * p.nv) * dvp;
            for (int b = 0; b < p.nv_perp; ++b) {
                const double vb = ((double)b + 0.5 - 0.5 * p.nv_perp) * dvq;
                if (dru) {
                    double h, dh;
                    D.marg2(va, vb, &h, &dh);
                    t.f0.push_back(h);
                    t.f0p.push_back(dh);
                } else {
                    const double g = std::exp(-(va * va + vb * vb) / two_vth2) / (kPi * two_vth2);
                    t.f0.push_back(g);
                    t.f0p.push_back(-va / (vth * vth) * g);
                }
                t.v.push_back(va); t.w.push_back(va * dvp * dvq); t.dV.push_back(dvp * dvq);
                t.speed.push_back(std::sqrt(va * va + vb * vb));
            }
        }
    } else if (p.vgrid == FDTD_VGRID_SPEED3D) {
        const double gam = vmax / p.nv;
        for (int k = 0; k < p.nv; ++k) {
            const double vk = ((double)k + 0.5) * gam;
            if (dru) {
                const double g = D.f(vk * vk);
                t.f0.push_back(g);
                t.f0p.push_back(-(kMe * kMe * vk * vk * vk / (D.eps0 * D.eps0)) * g);
            } else {
                const double g = std::exp(-vk * vk / two_vth2) / std::pow(kPi * two_vth2, 1.5);
                t.f0.push_back(g);
                t.f0p.push_back(-vk / (vth * vth) * g);
            }
            t.v.push_back(vk); t.w.push_back(4.0 * kPi / 3.0 * vk * vk * vk * gam);
            t.dV.push_back(4.0 * kPi * vk * vk * gam); t.speed.push_back(vk);
        }
    } else {
        return false;
    }
    // collision law (Eq. 23): nu = N s(v) |v|, N from the F0-weighted mean
    double num = 0.0, den = 0.0;
    for (size_t j = 0; j < t.v.size(); ++j) {
        const double sv = p.nu_model == FDTD_NU_TABLE ? table_sigma(p, t.speed[j]) * t.speed[j] : t.speed[j];
        t.sv.push_back(sv);
        num += sv * t.f0[j] * t.dV[j];
        den += t.f0[j] * t.dV[j];
    }
    t.mean_sv = num / den;
    for (size_t j = 0; j < t.v.size(); ++j) t.nu.push_back(node_nu(p, t, j, p.nu0));
    return true;
}

}  // namespace fp
