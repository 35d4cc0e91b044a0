// tables.cpp -- host FP64 construction of the sampling tables (Sec. 2.2).
//
// Nonlinear Compton (quantum synchrotron, the model the paper takes from
// EPOCH): emissivity F(eta, chi) = delta^2 y K_{2/3}(y) + (1 - delta) y
// Int_y^inf K_{5/3}, with delta = 2 chi / eta the photon energy fraction and
// y = 2 delta / (3 eta (1 - delta)).  Per eta row the table holds
//   h(eta)       = Int_0^inf F * 2/(2 + 3 eta y) d ln y      (= Int F/chi dchi)
//   CDF(eta, y_j) = Int_0^{y_j} (same integrand) / h(eta)
// and one extra row for eta -> 0, where the integrand tends to y Int_y K53.
//
// Bremsstrahlung: Eq. (1) with Tsai's Thomas-Fermi screening functions (the
// paper's Eqs. 3.38-3.41 reference), clamped at zero where the fit turns
// negative at the kinematic tip; sigma(E) integrates it from y_cut =
// photon_min / gamma to y_max = 1 - 1/gamma, and the CDF of sigma(y, E) is
// tabulated over s with y = y_cut (y_max / y_cut)^s.
//
// Bethe-Heitler pair production (Sec. 2.2: implemented like the bremsstrahlung):
// Tsai's DCS of the crossed process with the same fits, clamped at zero, integrated
// over the positron fraction x in [1/k, 1 - 1/k]; the CDF is tabulated linearly in x.
//
// Numerics (chosen independently of the test oracle): the Bessel integrals
// K_nu(x) = Int_0^inf exp(-x cosh t) cosh(nu t) dt and Int_x^inf K_{5/3} =
// Int_0^inf exp(-x cosh t) cosh(5t/3) / cosh t dt are evaluated by the
// trapezoidal rule, which converges geometrically for these even integrands
// analytic in |Im t| < pi/2; table cells use composite 8-point Gauss-Legendre
// on panels refined where the integrand varies fast.
#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace pe {
namespace {

const double GL_X[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
const double GL_W[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

template <class F>
double gauss8(const F& f, double a, double b) {
    double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < 4; ++i) s += GL_W[i] * (f(c - h * GL_X[i]) + f(c + h * GL_X[i]));
    return s * h;
}
template <class F>
double gauss8_panels(const F& f, double a, double b, int m) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += gauss8(f, a + (b - a) * k / m, a + (b - a) * (k + 1) / m);
    return s;
}

// trapezoid over t in [0, T] of exp(-x cosh t) * g(t), even integrand
template <class G>
double trap_bessel(double x, double nu, const G& g) {
    const double h = 0.2;
    // cut where exp(-x (cosh t - 1) + nu t) < 1e-22
    double T = 1.0;
    while (x * (std::cosh(T) - 1.0) - nu * T < 50.0) T += 0.5;
    double s = 0.5 * std::exp(-x) * g(0.0);
    for (double t = h; t <= T; t += h) s += std::exp(-x * std::cosh(t)) * g(t);
    return s * h;
}

double bessel_k23(double x) {
    return trap_bessel(x, 2.0 / 3.0, [](double t) { return std::cosh(2.0 * t / 3.0); });
}
double int_k53(double x) {
    return trap_bessel(x, 5.0 / 3.0, [](double t) { return std::cosh(5.0 * t / 3.0) / std::cosh(t); });
}

// integrand of the NCS CDF in ln y
double ncs_integrand(double eta, bool classical, double lny) {
    double y = std::exp(lny);
    if (y > 700.0) return 0.0;
    if (classical) return y * int_k53(y);
    double d = 3.0 * eta * y / (2.0 + 3.0 * eta * y);
    double F = d * d * y * bessel_k23(y) + (1.0 - d) * y * int_k53(y);
    return F * 2.0 / (2.0 + 3.0 * eta * y);
}

// one ln-y cell: panels so that each spans at most 0.5 in y and 0.2 in ln y
double ncs_cell(double eta, bool classical, double a, double b) {
    double ya = std::exp(a), yb = std::exp(b);
    int m = (int)std::ceil(std::max((yb - ya) / 0.5, (b - a) / 0.2));
    if (m < 1) m = 1;
    return gauss8_panels([&](double l) { return ncs_integrand(eta, classical, l); }, a, b, m);
}

void ncs_row(const pe_table_params& p, double eta, bool classical, double* row, double* total) {
    double lmin = std::log(p.y_min), lmax = std::log(p.y_max);
    double llo = lmin - 8.0 * std::log(10.0);           // y_lo = y_min * 1e-8
    // [0, y_lo]: integrand ~ y^(1/3), tail = 3 f(y_lo); [y_lo, y_min] numerically
    double cum = 3.0 * ncs_integrand(eta, classical, llo) + ncs_cell(eta, classical, llo, lmin);
    row[0] = cum;
    for (int j = 1; j < p.n_y; ++j) {
        double a = lmin + (lmax - lmin) * (j - 1) / (p.n_y - 1);
        double b = lmin + (lmax - lmin) * j / (p.n_y - 1);
        cum += ncs_cell(eta, classical, a, b);
        row[j] = cum;
    }
    *total = cum;
    for (int j = 0; j < p.n_y; ++j) row[j] /= cum;
    row[p.n_y - 1] = 1.0;
}

// ---- bremsstrahlung ---------------------------------------------------------
double coulomb_f(double Z) {
    double a2 = (kAlpha * Z) * (kAlpha * Z);
    return a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
}

struct Tsai {
    double Z, Z2, lnZ, f, z13, z23;
    explicit Tsai(double z) : Z(z), Z2(z * z), lnZ(std::log(z)), f(coulomb_f(z)), z13(std::cbrt(z)), z23(std::cbrt(z * z)) {}
    // y dsigma/dy in alpha r_e^2 (unclamped)
    double y_dcs(double gamma, double y) const {
        double q = 100.0 * y / (gamma * (1.0 - y));
        double g = q / z13, e = q / z23;
        double phi1 = 20.863 - 2.0 * std::log(1.0 + 0.55846 * 0.55846 * g * g)
                      - 4.0 * (1.0 - 0.6 * std::exp(-0.9 * g) - 0.4 * std::exp(-1.5 * g));
        double dphi = (2.0 / 3.0) / (1.0 + g * (6.5 + 6.0 * g));          // phi1 - phi2
        double psi1 = 28.340 - 2.0 * std::log(1.0 + 3.621 * 3.621 * e * e)
                      - 4.0 * (1.0 - 0.7 * std::exp(-8.0 * e) - 0.3 * std::exp(-29.2 * e));
        double dpsi = (2.0 / 3.0) / (1.0 + e * (40.0 + 400.0 * e));       // psi1 - psi2
        double a = (4.0 / 3.0) * (1.0 - y) + y * y;
        return a * (Z2 * (phi1 - (4.0 / 3.0) * lnZ - 4.0 * f) + Z * (psi1 - (8.0 / 3.0) * lnZ))
               + (2.0 / 3.0) * (1.0 - y) * (Z2 * dphi + Z * dpsi);
    }
};

// integral over s in [a, b] of max(y dsigma/dy, 0) * L with y = ycut exp(s L)
double brems_piece(const Tsai& ts, double gamma, double ycut, double L, double a, double b) {
    // breakpoints where 1 - y halves: the integrand is smooth in ln(1 - y)
    std::vector<double> br{a};
    for (int k = 1; k < 64; ++k) {
        double y = 1.0 - std::ldexp(1.0, -k);
        if (y <= ycut) continue;
        double s = std::log(y / ycut) / L;
        if (s > a && s < b) br.push_back(s);
        if (s >= b) break;
    }
    br.push_back(b);
    auto fn = [&](double s) {
        double y = ycut * std::exp(s * L);
        double v = ts.y_dcs(gamma, y);
        return v > 0.0 ? v * L : 0.0;
    };
    auto raw = [&](double s) { return ts.y_dcs(gamma, ycut * std::exp(s * L)); };
    double tot = 0.0;
    for (size_t k = 0; k + 1 < br.size(); ++k) {
        double lo = br[k], hi = br[k + 1];
        double flo = raw(lo), fhi = raw(hi);
        if ((flo < 0.0) != (fhi < 0.0)) {
            // clamp kink: bisect the sign change and integrate both sides
            double u = lo, v = hi;
            for (int it = 0; it < 200 && v - u > 1e-16 * (1.0 + std::fabs(u)); ++it) {
                double m = 0.5 * (u + v);
                if ((raw(m) < 0.0) == (flo < 0.0)) u = m; else v = m;
            }
            double r = 0.5 * (u + v);
            tot += gauss8_panels(fn, lo, r, 4) + gauss8_panels(fn, r, hi, 4);
        } else {
            tot += gauss8_panels(fn, lo, hi, 4);
        }
    }
    return tot;
}

void brems_row(const pe_table_params& p, const Tsai& ts, double gamma, double* row, double* sigma) {
    int n = p.n_s;
    double ycut = p.photon_min_mc2 / gamma, ymax = 1.0 - 1.0 / gamma;
    if (!(ycut < ymax)) {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (n - 1);
        *sigma = 0.0;
        return;
    }
    double L = std::log(ymax / ycut);
    double cum = 0.0;
    row[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        cum += brems_piece(ts, gamma, ycut, L, (double)(j - 1) / (n - 1), (double)j / (n - 1));
        row[j] = cum;
    }
    *sigma = cum;
    if (cum > 0.0) {
        for (int j = 0; j < n; ++j) row[j] /= cum;
        row[n - 1] = 1.0;
    } else {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (n - 1);
    }
}

// ---- Bethe-Heitler pair production -------------------------------------------
// Tsai's DCS of the crossed process with the same screening fits: photon k (m c^2),
// positron fraction x, screening variables 100 / (k x (1-x) Z^{1/3}), 100 / (k x (1-x)
// Z^{2/3}); d sigma / dx in alpha r_e^2 (unclamped).
double bh_dcs(const Tsai& ts, double k, double x) {
    double xx = x * (1.0 - x);
    double q = 100.0 / (k * xx);
    double g = q / ts.z13, e = q / ts.z23;
    double phi1 = 20.863 - 2.0 * std::log(1.0 + 0.55846 * 0.55846 * g * g)
                  - 4.0 * (1.0 - 0.6 * std::exp(-0.9 * g) - 0.4 * std::exp(-1.5 * g));
    double dphi = (2.0 / 3.0) / (1.0 + g * (6.5 + 6.0 * g));
    double psi1 = 28.340 - 2.0 * std::log(1.0 + 3.621 * 3.621 * e * e)
                  - 4.0 * (1.0 - 0.7 * std::exp(-8.0 * e) - 0.3 * std::exp(-29.2 * e));
    double dpsi = (2.0 / 3.0) / (1.0 + e * (40.0 + 400.0 * e));
    return (1.0 - (4.0 / 3.0) * xx) * (ts.Z2 * (phi1 - (4.0 / 3.0) * ts.lnZ - 4.0 * ts.f) + ts.Z * (psi1 - (8.0 / 3.0) * ts.lnZ))
           - (2.0 / 3.0) * xx * (ts.Z2 * dphi + ts.Z * dpsi);
}

// integral over s in [a, b] of max(dsigma/dx, 0) * span, x = xmin + s span: breakpoints
// where x or 1 - x halves (the screening varies with ln x near the ends), and the clamp
// kink bisected
double bh_piece(const Tsai& ts, double k, double xmin, double span, double a, double b) {
    std::vector<double> br{a};
    for (int e = 1; e < 64; ++e) {
        const double h = std::ldexp(1.0, -e);
        for (double xv : {h, 1.0 - h}) {
            double s = (xv - xmin) / span;
            if (s > a && s < b) br.push_back(s);
        }
        if (h < xmin) break;
    }
    br.push_back(b);
    std::sort(br.begin(), br.end());
    auto raw = [&](double s) { return bh_dcs(ts, k, xmin + s * span); };
    auto fn = [&](double s) {
        double v = raw(s);
        return v > 0.0 ? v * span : 0.0;
    };
    double tot = 0.0;
    for (size_t q = 0; q + 1 < br.size(); ++q) {
        double lo = br[q], hi = br[q + 1];
        if (!(hi > lo)) continue;
        double flo = raw(lo), fhi = raw(hi);
        if ((flo < 0.0) != (fhi < 0.0)) {
            double u = lo, v = hi;
            for (int it = 0; it < 200 && v - u > 1e-16 * (1.0 + std::fabs(u)); ++it) {
                double m = 0.5 * (u + v);
                if ((raw(m) < 0.0) == (flo < 0.0)) u = m; else v = m;
            }
            double r = 0.5 * (u + v);
            tot += gauss8_panels(fn, lo, r, 4) + gauss8_panels(fn, r, hi, 4);
        } else {
            tot += gauss8_panels(fn, lo, hi, 4);
        }
    }
    return tot;
}

void bh_row(const pe_table_params& p, const Tsai& ts, double k, double* row, double* sigma) {
    int n = p.n_s;
    if (!(k > 2.0)) {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (n - 1);
        *sigma = 0.0;
        return;
    }
    double xmin = 1.0 / k, span = 1.0 - 2.0 / k;
    double cum = 0.0;
    row[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        cum += bh_piece(ts, k, xmin, span, (double)(j - 1) / (n - 1), (double)j / (n - 1));
        row[j] = cum;
    }
    *sigma = cum;
    if (cum > 0.0) {
        for (int j = 0; j < n; ++j) row[j] /= cum;
        row[n - 1] = 1.0;
    } else {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (n - 1);
    }
}

template <class F>
void parallel_for(int n, const F& f) {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (nt > 64) nt = 64;
    if ((int)nt > n) nt = (unsigned)(n > 0 ? n : 1);
    std::vector<std::thread> th;
    for (unsigned k = 0; k < nt; ++k)
        th.emplace_back([&, k] {
            for (int i = (int)k; i < n; i += (int)nt) f(i);
        });
    for (auto& t : th) t.join();
}

}  // namespace

bool build_host_tables(const pe_table_params& p, HostTables& out, std::string* err) {
    out.p = p;
    out.Z.assign(p.Z, p.Z + p.n_Z);
    out.p.Z = nullptr;
    out.h.assign(p.n_eta, 0.0);
    out.cdf.assign((size_t)(p.n_eta + 1) * p.n_y, 0.0);
    out.sigma.assign((size_t)p.n_Z * p.n_E, 0.0);
    out.bcdf.assign((size_t)p.n_Z * p.n_E * p.n_s, 0.0);
    double le0 = std::log(p.eta_min), le1 = std::log(p.eta_max);
    double lg0 = std::log(p.gamma_min), lg1 = std::log(p.gamma_max);
    int n_ncs = p.n_eta + 1;
    int n_br = p.n_Z * p.n_E;
    std::vector<double> totals(n_ncs, 0.0);
    parallel_for(n_ncs + n_br, [&](int k) {
        if (k < n_ncs) {
            bool classical = (k == p.n_eta);
            double eta = classical ? 0.0 : std::exp(le0 + (le1 - le0) * k / (p.n_eta - 1));
            ncs_row(p, eta, classical, &out.cdf[(size_t)k * p.n_y], &totals[k]);
        } else {
            int b = k - n_ncs;
            int iz = b / p.n_E, i = b % p.n_E;
            Tsai ts(out.Z[iz]);
            double g = std::exp(lg0 + (lg1 - lg0) * i / (p.n_E - 1));
            brems_row(p, ts, g, &out.bcdf[((size_t)iz * p.n_E + i) * p.n_s], &out.sigma[(size_t)iz * p.n_E + i]);
        }
    });
    for (int i = 0; i < p.n_eta; ++i) out.h[i] = totals[i];
    out.classical_total = totals[p.n_eta];
    for (double v : out.h)
        if (!std::isfinite(v) || v <= 0.0) {
            if (err) *err = "NCS table build produced a non-positive h(eta)";
            return false;
        }
    return true;
}

}  // namespace pe

namespace pe {

void build_host_bh_tables(const HostTables& h, std::vector<double>& sigma, std::vector<double>& cdf) {
    const pe_table_params& p = h.p;
    const int nZ = (int)h.Z.size();
    sigma.assign((size_t)nZ * p.n_E, 0.0);
    cdf.assign((size_t)nZ * p.n_E * p.n_s, 0.0);
    const double l0 = std::log(2.0), l1 = std::log(p.gamma_max);
    parallel_for(nZ * p.n_E, [&](int b) {
        int iz = b / p.n_E, i = b % p.n_E;
        Tsai ts(h.Z[iz]);
        double k = std::exp(l0 + (l1 - l0) * i / (p.n_E - 1));
        bh_row(p, ts, k, &cdf[((size_t)iz * p.n_E + i) * p.n_s], &sigma[(size_t)iz * p.n_E + i]);
    });
}

}  // namespace pe

// ---- Breit-Wheeler tables ---------------------------------------------------------
// Pair production of a photon in a locally constant crossed field: per unit positron
// energy fraction x, G(chi, x) = (x/(1-x) + (1-x)/x) K_{2/3}(xi) + int_xi^inf K_{1/3},
// xi = 2 / (3 chi x (1 - x)); the rate is alpha (m c^2/hbar)(m c^2/(hbar omega)) T(chi),
// T = (1/(sqrt 3 pi)) int_0^1 G dx.
namespace pe {
namespace {

// trapezoid over t of exp(-x cosh t) g(t) with a step small against the width 1/sqrt(x) of
// the integrand at large x (the error falls as exp(-2 pi^2 / (x h^2)))
template <class G>
double trap_bessel_fine(double x, double nu, const G& g) {
    const double h = std::min(0.2, 0.5 / std::sqrt(x));
    double T = h;
    while (x * (std::cosh(T) - 1.0) - nu * T < 50.0) T += h;
    double s = 0.5 * std::exp(-x) * g(0.0);
    for (int k = 1; k * h <= T; ++k) {
        const double t = k * h;
        s += std::exp(-x * std::cosh(t)) * g(t);
    }
    return s * h;
}

double bw_G(double chi, double x) {
    if (!(x > 0.0) || !(x < 1.0)) return 0.0;
    const double xi = 2.0 / (3.0 * chi * x * (1.0 - x));
    if (xi > 700.0) return 0.0;
    const double k23 = trap_bessel_fine(xi, 2.0 / 3.0, [](double t) { return std::cosh(2.0 * t / 3.0); });
    const double ik13 = trap_bessel_fine(xi, 1.0 / 3.0, [](double t) { return std::cosh(t / 3.0) / std::cosh(t); });
    return (x / (1.0 - x) + (1.0 - x) / x) * k23 + ik13;
}

// cumulative int G dx over the cells of the node grid x_j = (1 - cos(pi s_j))/2, s_j = j/(n-1),
// integrated in s (dx = (pi/2) sin(pi s) ds), two 8-point Gauss panels per cell
void bw_row(double chi, int n, double* row, double* T) {
    constexpr double kPi = 3.14159265358979323846;
    const auto f = [chi](double s) {
        return bw_G(chi, 0.5 * (1.0 - std::cos(kPi * s))) * 0.5 * kPi * std::sin(kPi * s);
    };
    double cum = 0.0;
    row[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        cum += gauss8_panels(f, (double)(j - 1) / (n - 1), (double)j / (n - 1), 2);
        row[j] = cum;
    }
    *T = cum / (std::sqrt(3.0) * kPi);
    for (int j = 0; j < n; ++j) row[j] = cum > 0.0 ? row[j] / cum : (double)j / (n - 1);
}

}  // namespace

void build_host_bw_tables(int n_chi, double chi_min, double chi_max, int n_x, double* T, double* cdf) {
    const double l0 = std::log(chi_min), l1 = std::log(chi_max);
    parallel_for(n_chi, [&](int i) {
        const double chi = std::exp(l0 + (l1 - l0) * i / (n_chi - 1));
        bw_row(chi, n_x, cdf + (size_t)i * n_x, T + i);
    });
}

}  // namespace pe
