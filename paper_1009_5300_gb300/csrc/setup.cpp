// Host-side FP64 set-up: FD weights, electrode channels and self-energy per
// lateral mode, incident sources, lateral FFT plans and projector tables.
//
// Electrode channels.  In a flat jellium electrode the lateral plane waves
// exp(i G_nu . r) decouple Eq. 2 into one recurrence per mode nu,
//     (E - eps_perp) psi_k + (1 / (2 h_z^2)) sum_{|n| <= N_f} w_|n| psi_{k+n} = 0.
// With psi_k = lambda^k and u = (lambda + 1/lambda) / 2, lambda^n + lambda^-n =
// 2 T_n(u) (Chebyshev), so the 2 N_f roots come in pairs (lambda, 1/lambda)
// over the N_f roots u of the real degree-N_f polynomial
//     2 h_z^2 (E - eps_perp) + w_0 + 2 sum_n w_n T_n(u) = 0.
// For N_f = 1 this is u = -chi with chi of Eq. 9 and lambda = exp(i k_z h_z)
// of Eq. 8.5.  Of each pair the right-going root is kept: |lambda| < 1, or
// |lambda| = 1 with positive group velocity.
//
// Self-energy per mode (Eqs. 17-1/17-2 in the lateral Fourier basis): with
// depth d = 0 .. N_f-1 inward from the outermost plane and electrode planes
// e = 1 .. N_f outward, Sigma~ = -K Q_out Q_in^{-1}, K[d][e] = w_{d+e} / (2 h_z^2),
// Q_in[d][j] = lambda_j^-d, Q_out[e][j] = lambda_j^e.  Columns are scaled by
// lambda_j^(N_f-1) (which cancels in the product) to keep every entry <= 1.
// For N_f = 1: Sigma~ = -exp(i k_z h_z) / (2 h_z^2) (Eq. 18-2).
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <atomic>
#include <sstream>
#include <thread>

namespace iobm {

constexpr int kMaxNfHost = 4;

std::vector<double> fd_weights(int nf) {
    const int n = nf + 1;
    std::vector<long double> M((size_t)n * n), b(n);
    for (int m = 0; m < n; ++m) {
        M[(size_t)m * n + 0] = (m == 0) ? 1.0L : 0.0L;
        for (int j = 1; j <= nf; ++j) M[(size_t)m * n + j] = 2.0L * std::pow((long double)j, 2 * m);
        b[m] = (m == 1) ? 2.0L : 0.0L;
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)piv * n + c])) piv = r;
        for (int j = 0; j < n; ++j) std::swap(M[(size_t)c * n + j], M[(size_t)piv * n + j]);
        std::swap(b[c], b[piv]);
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const long double f = M[(size_t)r * n + c] / M[(size_t)c * n + c];
            for (int j = 0; j < n; ++j) M[(size_t)r * n + j] -= f * M[(size_t)c * n + j];
            b[r] -= f * b[c];
        }
    }
    std::vector<double> w(n);
    for (int c = 0; c < n; ++c) w[c] = (double)(b[c] / M[(size_t)c * n + c]);
    return w;
}

// a / b by the textbook formula: the library operator guards against overflow by
// scaling, which the moderate operands of the root finder never need
static inline cd cdiv(cd a, cd b) {
    const double d = b.real() * b.real() + b.imag() * b.imag();
    return cd((a.real() * b.real() + a.imag() * b.imag()) / d,
              (a.imag() * b.real() - a.real() * b.imag()) / d);
}

// Roots of sum_k a[k] u^k (real coefficients, a.back() != 0) by the Aberth-Ehrlich
// simultaneous iteration, then a Newton polish on the same polynomial.  guess
// (may be null): starting points, e.g. the roots of a nearby polynomial; if they
// do not converge within a few dozen steps the iteration restarts from points on
// a circle inside the Cauchy bound.
static std::vector<cd> poly_roots(const std::vector<double>& a, const std::vector<cd>* guess) {
    const int n = (int)a.size() - 1;
    std::vector<cd> z(n);
    if (n == 1) {
        z[0] = cd(-a[0] / a[1], 0.0);
        return z;
    }
    std::vector<double> c(a.size());
    for (int k = 0; k <= n; ++k) c[k] = a[k] / a[n];
    auto eval = [&](cd x, cd& p, cd& dp) {
        p = cd(1.0, 0.0);
        dp = cd(0.0, 0.0);
        for (int k = n - 1; k >= 0; --k) {
            dp = dp * x + p;
            p = p * x + c[k];
        }
    };
    auto aberth = [&](int max_it) {
        for (int it = 0; it < max_it; ++it) {
            double maxstep = 0.0;
            for (int k = 0; k < n; ++k) {
                cd p, dp;
                eval(z[k], p, dp);
                if (p == cd(0.0, 0.0)) continue;
                const cd ratio = cdiv(p, dp);
                cd s(0.0, 0.0);
                for (int j = 0; j < n; ++j)
                    if (j != k) s += cdiv(1.0, z[k] - z[j]);
                const cd w = cdiv(ratio, 1.0 - ratio * s);
                z[k] -= w;
                maxstep = std::max(maxstep, std::abs(w) / std::max(1.0, std::abs(z[k])));
            }
            if (!(maxstep >= 1e-13)) return maxstep == maxstep;   // converged (not NaN)
        }
        return false;
    };
    auto polish = [&]() {   // Newton steps on the same polynomial
        for (int k = 0; k < n; ++k) {
            for (int it = 0; it < 3; ++it) {
                cd p, dp;
                eval(z[k], p, dp);
                if (dp == cd(0.0, 0.0)) break;
                z[k] -= p / dp;
            }
        }
    };
    auto distinct = [&](double tol) {
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < k; ++j)
                if (!(std::abs(z[k] - z[j]) > tol * std::max(1.0, std::abs(z[k])))) return false;
        return true;
    };
    if (guess && (int)guess->size() == n) {
        z = *guess;
        if (distinct(1e-12) && aberth(40)) {
            polish();
            // two starting points drawn to one root would leave another root unfound
            if (distinct(1e-10)) return z;
        }
    }
    double R = 0.0;
    for (int k = 0; k < n; ++k) R = std::max(R, std::fabs(c[k]));
    R = 1.0 + R;   // Cauchy bound
    for (int k = 0; k < n; ++k) z[k] = std::polar(0.7 * R, 2.0 * M_PI * k / n + 0.4);
    aberth(80);
    polish();
    return z;
}

static double velocity(double theta, const std::vector<double>& w, double hz) {
    double v = 0.0;
    for (int n = 1; n < (int)w.size(); ++n) v += n * w[n] * std::sin(n * theta);
    return v / hz;
}

static inline int nu_of_index(int i, int n) { return i - n / 2; }          // canonical nu
static inline int bin_of_nu(int nu, int n) { return ((nu % n) + n) % n; }   // FFT bin

namespace {

// Everything the solver needs about one lateral mode depends on E - eps_perp
// only, so it is computed once per distinct eps_perp.
struct ModeSolution {
    bool open = false;
    double vel = 0.0;
    cd lam_in;
    cd sigma[kMaxNfHost * kMaxNfHost];
    cd pc[kPcStride];
    cd mrow[kMaxNfHost];
    cd btilde[kMaxNfHost];
};

// Gauss-Jordan inverse of an n x n complex matrix (row-major, n <= 4), partial pivoting.
bool cinv_small(cd* A, int n) {
    cd I[kMaxNfHost * kMaxNfHost];
    for (int i = 0; i < n * n; ++i) I[i] = 0.0;
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[r * n + c]) > std::abs(A[piv * n + c])) piv = r;
        if (std::abs(A[piv * n + c]) == 0.0) return false;
        for (int j = 0; j < n; ++j) {
            std::swap(A[c * n + j], A[piv * n + j]);
            std::swap(I[c * n + j], I[piv * n + j]);
        }
        const cd inv = cdiv(1.0, A[c * n + c]);
        for (int j = 0; j < n; ++j) {
            A[c * n + j] *= inv;
            I[c * n + j] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const cd f = A[r * n + c];
            if (f == cd(0.0, 0.0)) continue;
            for (int j = 0; j < n; ++j) {
                A[r * n + j] -= f * A[c * n + j];
                I[r * n + j] -= f * I[c * n + j];
            }
        }
    }
    for (int i = 0; i < n * n; ++i) A[i] = I[i];
    return true;
}

cd ipow(cd x, int n) {
    cd r(1.0, 0.0);
    if (n < 0) {
        x = cdiv(1.0, x);
        n = -n;
    }
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

// Roots, self-energy, preconditioner factors, projection row and source of
// one lateral mode with E - eps_perp = dE.  Returns 0 or 9 (more than one
// propagating root / singular block).
// roots: in, the u-roots of a nearby mode as starting points (may be empty); out,
// this mode's u-roots.
int solve_mode(double dE, int nf, double hz, const std::vector<double>& w,
               const std::vector<std::vector<double>>& tc, const double* K, bool want_sigma,
               ModeSolution& m, std::string& msg, std::vector<cd>& roots) {
    std::vector<double> a(nf + 1, 0.0);
    a[0] = 2.0 * hz * hz * dE + w[0];
    for (int n = 1; n <= nf; ++n)
        for (int k = 0; k <= n; ++k) a[k] += 2.0 * w[n] * tc[n][k];
    const std::vector<cd> us = poly_roots(a, roots.empty() ? nullptr : &roots);
    roots = us;
    cd lam[kMaxNfHost];
    int prop = -1;
    for (int j = 0; j < nf; ++j) {
        cd u = us[j];
        if (std::fabs(u.imag()) <= 1e-12 * std::max(1.0, std::abs(u))) u = cd(u.real(), 0.0);
        if (u.imag() == 0.0 && std::fabs(u.real()) < 1.0) {
            const double th = std::acos(u.real());
            const double v = velocity(th, w, hz);
            lam[j] = std::polar(1.0, (v > 0.0 ? 1.0 : -1.0) * th);
            if (prop >= 0) {
                msg = "more than one propagating root in one lateral mode";
                return 9;
            }
            prop = j;
            m.vel = std::fabs(v);
        } else {
            const cd sq = std::sqrt(u * u - 1.0);
            const cd l1 = u - sq, l2 = u + sq;
            lam[j] = (std::abs(l1) < std::abs(l2)) ? l1 : l2;
        }
    }
    // scaled Q_in[d][j] = lam_j^(nf-1-d); Q_out[e-1][j] = lam_j^(e+nf-1)
    cd Qinv[kMaxNfHost * kMaxNfHost], Qout[kMaxNfHost * kMaxNfHost];
    for (int j = 0; j < nf; ++j) {
        cd p = 1.0;
        cd pw[2 * kMaxNfHost];
        for (int k = 0; k < 2 * nf; ++k) {
            pw[k] = p;
            p *= lam[j];
        }
        for (int d = 0; d < nf; ++d) Qinv[d * nf + j] = pw[nf - 1 - d];
        for (int e = 1; e <= nf; ++e) Qout[(e - 1) * nf + j] = pw[e + nf - 1];
    }
    if (!cinv_small(Qinv, nf)) {
        msg = "singular Bloch-state matrix";
        return 9;
    }
    // S = -K Qout Qinv
    cd KQ[kMaxNfHost * kMaxNfHost], S[kMaxNfHost * kMaxNfHost];
    for (int d = 0; d < nf; ++d)
        for (int j = 0; j < nf; ++j) {
            cd acc = 0.0;
            for (int e = 0; e < nf; ++e) acc += K[d * nf + e] * Qout[e * nf + j];
            KQ[d * nf + j] = acc;
        }
    for (int d = 0; d < nf; ++d)
        for (int dp = 0; dp < nf; ++dp) {
            cd acc = 0.0;
            for (int j = 0; j < nf; ++j) acc -= KQ[d * nf + j] * Qinv[j * nf + dp];
            S[d * nf + dp] = acc;
        }
    for (int i = 0; i < nf * nf; ++i) m.sigma[i] = S[i];
    if (want_sigma) {
        // Free-propagator preconditioner of this mode: E - eps_perp - T_z - Sigma at
        // both ends.  Gaussian elimination from the left end keeps the left
        // self-energy pattern on the leading block (eliminating one more plane of
        // a semi-infinite lead reproduces the lead), so the band factors are the
        // same on every row of the first nz - nf planes:
        //   u_j = T[0][j] - S[0][j],  l_j = (T[j][0] - S[j][0]) / u_0,
        // and the last nf planes form the block T - S - flip(S).
        auto Tm = [&](int i, int j) {
            const int n = std::abs(i - j);
            double v = (n <= nf) ? w[n] / (2.0 * hz * hz) : 0.0;
            if (i == j) v += dE;
            return cd(v, 0.0);
        };
        cd u[kMaxNfHost + 1];
        for (int j = 0; j <= nf; ++j) u[j] = Tm(0, j) - (j < nf ? S[j] : cd(0.0, 0.0));
        for (int j = 1; j <= nf; ++j)
            m.pc[j - 1] = (Tm(j, 0) - (j < nf ? S[j * nf] : cd(0.0, 0.0))) / u[0];
        for (int j = 0; j <= nf; ++j) m.pc[nf + j] = u[j];
        cd S2[kMaxNfHost * kMaxNfHost];
        for (int i = 0; i < nf; ++i)
            for (int j = 0; j < nf; ++j)
                S2[i * nf + j] = Tm(i, j) - S[i * nf + j] - S[(nf - 1 - i) * nf + (nf - 1 - j)];
        if (!cinv_small(S2, nf)) {
            msg = "singular end block of the free-propagator preconditioner";
            return 9;
        }
        for (int i = 0; i < nf * nf; ++i) m.pc[2 * nf + 1 + i] = S2[i];
    }
    m.open = prop >= 0;
    if (m.open) {
        const cd li = lam[prop];
        m.lam_in = li;
        const cd scale = ipow(li, nf - 1);
        for (int d = 0; d < nf; ++d) m.mrow[d] = scale * Qinv[prop * nf + d];
        for (int d = 0; d < nf; ++d) {
            cd b(0.0, 0.0);
            for (int e = 1; e <= nf; ++e) b -= K[d * nf + (e - 1)] * ipow(li, -e);
            for (int dp = 0; dp < nf; ++dp) b -= S[d * nf + dp] * ipow(li, dp);
            m.btilde[d] = b;
        }
    }
    return 0;
}

}  // namespace

int build_mode_tables(int nx, int ny, double hx, double hy, double hz, int nf, double E,
                      bool want_sigma, ModeTables& out, std::string& msg, double kappa_x,
                      double kappa_y) {
    const std::vector<double> w = fd_weights(nf);
    const double two_pi = 2.0 * M_PI;
    // lateral dispersion at G_nu + kappa (Eq. 8 with the lateral Bloch vector)
    auto eps1d = [&](int nu, int n, double h, double kappa) {
        const double G = two_pi * nu / (n * h) + kappa;
        double s = w[0];
        for (int k = 1; k <= nf; ++k) s += 2.0 * w[k] * std::cos(k * G * h);
        return -0.5 * s / (h * h);
    };
    double top_s = w[0];
    for (int k = 1; k <= nf; ++k) top_s += 2.0 * w[k] * ((k & 1) ? -1.0 : 1.0);
    const double band_top = -0.5 * top_s / (hz * hz);

    // Chebyshev coefficients T_n(u) = sum_k tc[n][k] u^k
    std::vector<std::vector<double>> tc(nf + 1, std::vector<double>(nf + 1, 0.0));
    tc[0][0] = 1.0;
    if (nf >= 1) tc[1][1] = 1.0;
    for (int n = 2; n <= nf; ++n)
        for (int k = 0; k <= nf; ++k)
            tc[n][k] = (k > 0 ? 2.0 * tc[n - 1][k - 1] : 0.0) - tc[n - 2][k];

    double K[kMaxNfHost * kMaxNfHost] = {};
    for (int d = 0; d < nf; ++d)
        for (int e = 1; e <= nf; ++e)
            if (d + e <= nf) K[d * nf + (e - 1)] = w[d + e] / (2.0 * hz * hz);

    out = ModeTables();
    out.E = E;
    if (want_sigma) {
        out.sigma.assign((size_t)nx * ny * nf * nf, cd(0.0, 0.0));
        out.pc.assign((size_t)nx * ny * kPcStride, cd(0.0, 0.0));
    }
    out.eperp_bin.assign((size_t)nx * ny, 0.0);
    std::vector<double> ex(nx), ey(ny);
    for (int ix = 0; ix < nx; ++ix) ex[ix] = eps1d(nu_of_index(ix, nx), nx, hx, kappa_x);
    for (int iy = 0; iy < ny; ++iy) ey[iy] = eps1d(nu_of_index(iy, ny), ny, hy, kappa_y);
    // distinct lateral energies (the dispersion is even in nu, and symmetric in
    // x <-> y on square cells), each solved once
    std::vector<double> eperp((size_t)nx * ny);
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) eperp[(size_t)iy * nx + ix] = ex[ix] + ey[iy];
    std::vector<double> uniq(eperp);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    std::vector<ModeSolution> sol(uniq.size());
    std::vector<cd> roots;   // the previous (nearest smaller) eps_perp's roots start the next
    for (size_t u = 0; u < uniq.size(); ++u) {
        if (std::fabs(E - uniq[u]) < 1e-9 || std::fabs(E - uniq[u] - band_top) < 1e-9) {
            std::ostringstream os;
            os << "energy " << E << " Ha lies within 1e-9 Ha of the threshold of a lateral mode "
               << "with eps_perp = " << uniq[u] << " Ha";
            msg = os.str();
            return 2;
        }
        const int rc = solve_mode(E - uniq[u], nf, hz, w, tc, K, want_sigma, sol[u], msg, roots);
        if (rc) return rc;
    }
    for (int iy = 0; iy < ny; ++iy) {
        const int nuy = nu_of_index(iy, ny);
        for (int ix = 0; ix < nx; ++ix) {
            const int nux = nu_of_index(ix, nx);
            const int canon = iy * nx + ix;
            const size_t u = std::lower_bound(uniq.begin(), uniq.end(), eperp[canon]) - uniq.begin();
            const ModeSolution& m = sol[u];
            const int kx = bin_of_nu(nux, nx), ky = bin_of_nu(nuy, ny);
            out.eperp_bin[(size_t)ky * nx + kx] = eperp[canon];
            if (want_sigma) {
                cd* dst = &out.sigma[((size_t)ky * nx + kx) * nf * nf];
                for (int i = 0; i < nf * nf; ++i) dst[i] = m.sigma[i];
                cd* pc = &out.pc[((size_t)ky * nx + kx) * kPcStride];
                for (int i = 0; i < kPcStride; ++i) pc[i] = m.pc[i];
            }
            if (m.open) {
                out.open_canon.push_back(canon);
                out.open_kx.push_back(kx);
                out.open_ky.push_back(ky);
                out.open_nux.push_back(nux);
                out.open_nuy.push_back(nuy);
                out.vel.push_back(m.vel);
                out.lam_in.push_back(m.lam_in);
                for (int d = 0; d < nf; ++d) out.mrow.push_back(m.mrow[d]);
                for (int d = 0; d < nf; ++d) out.btilde.push_back(m.btilde[d]);
            }
        }
    }
    out.nopen = (int)out.open_canon.size();
    // partner channel (-nu) of every open channel; at kappa = 0 the lateral dispersion
    // is even in nu (at kappa != 0 the partner is a channel of -kappa: none is recorded)
    out.open_partner.assign(out.nopen, -1);
    if (kappa_x != 0.0 || kappa_y != 0.0) return 0;
    for (int c = 0; c < out.nopen; ++c) {
        const int bx = bin_of_nu(-out.open_nux[c], nx), by = bin_of_nu(-out.open_nuy[c], ny);
        for (int d = 0; d < out.nopen; ++d)
            if (out.open_kx[d] == bx && out.open_ky[d] == by) out.open_partner[c] = d;
        if (out.open_partner[c] < 0) {
            msg = "open channel without a -nu partner";
            return 9;
        }
    }
    return 0;
}

int build_mode_tables_many(int nx, int ny, double hx, double hy, double hz, int nf, const double* E,
                           int nE, bool want_sigma, std::vector<ModeTables>& out, std::string& msg,
                           double kappa_x, double kappa_y) {
    out.assign(nE, ModeTables());
    std::vector<int> rc(nE, 0);
    std::vector<std::string> msgs(nE);
    const int nth = std::max(1, std::min<int>(nE, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next(0);
    auto work = [&]() {
        for (int e = next++; e < nE; e = next++)
            rc[e] = build_mode_tables(nx, ny, hx, hy, hz, nf, E[e], want_sigma, out[e], msgs[e],
                                      kappa_x, kappa_y);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int e = 0; e < nE; ++e)
        if (rc[e]) {
            msg = msgs[e];
            return rc[e];
        }
    return 0;
}

void hermitian_eigenvalues(const std::vector<std::complex<double>>& m, int n, std::vector<double>& w) {
    const int N = 2 * n;
    std::vector<double> a((size_t)N * N, 0.0);
    auto at = [&](int i, int j) -> double& { return a[(size_t)i * N + j]; };
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            const std::complex<double> v = (i == j) ? std::complex<double>(m[(size_t)i * n + i].real(), 0.0)
                                                    : m[(size_t)i * n + j];
            // [[X, -Y], [Y, X]] with m = X + iY, X symmetric, Y antisymmetric
            at(i, j) = at(j, i) = v.real();
            at(n + i, n + j) = at(n + j, n + i) = v.real();
            at(n + i, j) = v.imag();
            at(j, n + i) = v.imag();
            at(i, n + j) = -v.imag();
            at(n + j, i) = -v.imag();
        }
    double scale = 0.0;
    for (double v : a) scale += v * v;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) off += at(i, j) * at(i, j);
        if (off <= 1e-30 * scale || off == 0.0) break;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q) {
                const double apq = at(p, q);
                if (apq == 0.0) continue;
                const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < N; ++k) {   // rotate columns p, q
                    const double akp = at(k, p), akq = at(k, q);
                    at(k, p) = c * akp - s * akq;
                    at(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < N; ++k) {   // and rows p, q
                    const double apk = at(p, k), aqk = at(q, k);
                    at(p, k) = c * apk - s * aqk;
                    at(q, k) = s * apk + c * aqk;
                }
            }
    }
    std::vector<double> d(N);
    for (int i = 0; i < N; ++i) d[i] = at(i, i);
    std::sort(d.begin(), d.end(), [](double x, double y) { return x > y; });
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = 0.5 * (d[2 * i] + d[2 * i + 1]);   // each value appears twice
}

bool fft_plan(int n, std::vector<int>& radices) {
    radices.clear();
    if (n < 1) return false;
    static const int order[] = {4, 2, 3, 5};
    for (int r : order) {
        while (n % r == 0) {
            radices.push_back(r);
            n /= r;
        }
    }
    return n == 1;
}

int build_projectors(int nproj, const int64_t* row_ptr, const int32_t* idx, const double* val,
                     const double* coupling, int nx, int ny, int nz, int nf, ProjTables& out,
                     std::string& msg) {
    out = ProjTables();
    out.nproj = nproj;
    if (nproj == 0) {
        out.pptr.assign(1, 0);
        out.uptr.assign(1, 0);
        return 0;
    }
    if (!row_ptr || !idx || !val || !coupling || nproj < 0) {
        msg = "projector arrays are NULL";
        return 1;
    }
    const long long plane = (long long)nx * ny;
    const long long npts = plane * nz;
    if (row_ptr[0] != 0) {
        msg = "projector row_ptr[0] must be 0";
        return 1;
    }
    struct Entry { int g, p; double v; };
    std::vector<Entry> all;
    out.pptr.assign(nproj + 1, 0);
    for (int p = 0; p < nproj; ++p) {
        const int64_t b = row_ptr[p], e = row_ptr[p + 1];
        if (e < b || e - b > (int64_t)npts) {
            msg = "projector row_ptr is not non-decreasing";
            return 1;
        }
        if (!std::isfinite(coupling[p])) {
            msg = "non-finite projector coupling";
            return 1;
        }
        std::vector<int> seen;
        for (int64_t i = b; i < e; ++i) {
            const long long g = idx[i];
            if (g < 0 || g >= npts) {
                msg = "projector index outside the grid";
                return 1;
            }
            if (!std::isfinite(val[i])) {
                msg = "non-finite projector value";
                return 1;
            }
            const long long k = g / plane;
            if (k < nf || k >= nz - nf) {
                std::ostringstream os;
                os << "projector " << p << " reaches plane " << k << " (the self-energy acts on planes < "
                   << nf << " and >= " << nz - nf << ")";
                msg = os.str();
                return 3;
            }
            out.pidx.push_back((int)g);
            out.pval.push_back(val[i]);
            all.push_back({(int)g, p, val[i]});
            seen.push_back((int)g);
        }
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
            msg = "projector lists a grid point twice";
            return 1;
        }
        out.pptr[p + 1] = (int)out.pidx.size();
        out.coupling.push_back(coupling[p]);
    }
    std::stable_sort(all.begin(), all.end(), [](const Entry& a, const Entry& b) {
        return a.g != b.g ? a.g < b.g : a.p < b.p;
    });
    out.uptr.push_back(0);
    for (size_t i = 0; i < all.size(); ++i) {
        if (i == 0 || all[i].g != all[i - 1].g) {
            if (i > 0) out.uptr.push_back((int)i);
            out.uidx.push_back(all[i].g);
        }
        out.uproj.push_back(all[i].p);
        out.uval.push_back(all[i].v);
    }
    out.uptr.push_back((int)all.size());
    if (all.empty()) out.uptr.assign(1, 0);
    return 0;
}

}  // namespace iobm
