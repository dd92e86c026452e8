// Host-side FP64 set-up of the electrode channels (per energy), the lateral FFT
// plans and the projector tables.  Plain C++ (no CUDA), compiled by the host
// compiler.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace iobm {

using cd = std::complex<double>;

// FD second-derivative weights w_0 .. w_nf of Eq. 1 (c_{mu,n} = w_|n| / h_mu^2).
std::vector<double> fd_weights(int nf);

struct ModeTables {
    double E = 0.0;
    int nopen = 0;
    std::vector<int> open_canon;       // canonical mode index (nu_y major) of each open channel
    std::vector<int> open_kx, open_ky; // FFT bins of each open channel
    std::vector<int> open_nux, open_nuy;
    std::vector<double> vel;           // group velocity of each open channel
    std::vector<cd> lam_in;            // propagating right-going root of each open channel
    std::vector<cd> mrow;              // [nopen][nf]: t = sum_d mrow[d] psi~(depth d)
    std::vector<cd> btilde;            // [nopen][nf]: incident source coefficients (Eq. 7)
    std::vector<int> open_partner;     // open-list index of the channel with lateral index -nu
    std::vector<cd> sigma;             // [ky][kx][nf][nf] Sigma~ in FFT-bin order
    // free-propagator preconditioner per FFT bin: banded LU of E - T - H~ for the
    // mode (constant factors l_1..l_nf, u_0..u_nf and the inverse of the last
    // nf x nf Schur block), [ky][kx][kPcStride]
    std::vector<cd> pc;
    std::vector<double> eperp_bin;     // [ky][kx] lateral energy eps_perp of each FFT bin
};

constexpr int kPcStride = 25;   // nf + (nf + 1) + nf * nf for nf = 4

// Builds the tables of energy E at lateral Bloch vector (kappa_x, kappa_y) (modes
// G_nu + kappa).  Returns 0, or 2 (IOBM_E_THRESHOLD) when E is within 1e-9 Ha of a
// channel edge, or 9 when a mode has more than one propagating right-going root.
// `msg` receives a one-line reason.  open_partner (the -nu channel) is filled at
// kappa = 0 only.
int build_mode_tables(int nx, int ny, double hx, double hy, double hz, int nf, double E,
                      bool want_sigma, ModeTables& out, std::string& msg, double kappa_x = 0.0,
                      double kappa_y = 0.0);

// The tables of several energies, built in parallel host threads.
int build_mode_tables_many(int nx, int ny, double hx, double hy, double hz, int nf, const double* E,
                           int nE, bool want_sigma, std::vector<ModeTables>& out, std::string& msg,
                           double kappa_x = 0.0, double kappa_y = 0.0);

// Radix plan of a lateral FFT length (radices 4, 2, 3, 5); false if n has
// another prime factor.
bool fft_plan(int n, std::vector<int>& radices);

struct ProjTables {
    int nproj = 0;
    std::vector<int> pptr, pidx;
    std::vector<double> pval, coupling;
    std::vector<int> uidx, uptr, uproj;
    std::vector<double> uval;
};

// Eigenvalues (descending) of the n x n complex Hermitian matrix m (row-major,
// only the upper triangle is read): cyclic Jacobi rotations on its real
// symmetric 2n x 2n embedding [[Re m, -Im m], [Im m, Re m]], whose spectrum is
// that of m with every eigenvalue twice.
void hermitian_eigenvalues(const std::vector<std::complex<double>>& m, int n, std::vector<double>& w);

// Validates and converts the CSR projectors.  Returns 0, 1 (IOBM_E_ARG) or
// 3 (IOBM_E_PROJ_BOUNDARY).
int build_projectors(int nproj, const int64_t* row_ptr, const int32_t* idx, const double* val,
                     const double* coupling, int nx, int ny, int nz, int nf, ProjTables& out,
                     std::string& msg);

}  // namespace iobm
