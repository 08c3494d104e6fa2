// Host FP64 numerics for the FTK plan: Gauss--Jacobi(0,1) rules, a symmetric
// eigensolver, a one-sided Jacobi SVD and the per-order operator SVD of
// J_l(x y) (Section 4.5, eq. Jsvd). No LAPACK: everything is written here.
#pragma once

#include <vector>

namespace ftk {

// Gauss--Jacobi rule with weight (1 - t)^alpha (1 + t)^beta on [-1, 1],
// by the Golub--Welsch method (eigenpairs of the Jacobi matrix).
void gauss_jacobi(int n, double alpha, double beta, std::vector<double>& t, std::vector<double>& w);

// Eigen-decomposition of a dense symmetric n x n matrix (row-major, destroyed)
// by cyclic Jacobi rotations: A = V diag(e) V^T, eigenvectors in columns of V.
void symmetric_eigen(int n, std::vector<double>& A, std::vector<double>& e, std::vector<double>& V);

// One-sided (Hestenes) Jacobi SVD of a dense m x n matrix (row-major), m >= n:
// A = U diag(s) V^T with s descending, U m x n, V n x n (row-major).
void svd_jacobi(int m, int n, const std::vector<double>& A, std::vector<double>& U,
                std::vector<double>& s, std::vector<double>& V);

// Operator SVD of J_l(x y) on x in [0, X] (weight x dx) by y in [0, 1] (weight
// y dy), discretized by Nystrom on Gauss--Jacobi(0,1) nodes.
//
// With CTF defocus values tau_b (Section 7.1) the kernel is J_l(x y) C_b(y),
// C_b(y) = -sin(pi tau_b y^2 + phase) (y = k / K), factorized jointly over the rows
// (x, tau_b) (weight x dx / n_tau) and y: J_l(x y) C_b(y) = sum U(x, b) Sigma V(y).
//
// With a spectral weight (the alternative k weights of Section 4.5) the norm over y is
// rho(y) y dy, rho(y) = exp(-decay y^2) decay / (1 - exp(-decay)) (unit mean over the
// disk): the SVD is that of J_l(x y) C_b(y) sqrt(rho(y)) in the plain weights, and
// V = Vtilde / sqrt(rho), so that U Sigma V still reconstructs J_l(x y) C_b(y).
struct ModalSVD {
  int l = 0;
  int nq = 0;
  double X = 0;
  std::vector<double> taus;             // CTF defocus values (empty: no CTF)
  double phase = 0;                     // CTF phase offset
  double decay = 0;                     // spectral weight exponent (0: plain weights)
  std::vector<double> sigma;            // all singular values, descending
  std::vector<double> xq, sqwx;         // x nodes, sqrt of weights
  std::vector<double> yq, sqwy;         // y nodes, sqrt of weights
  std::vector<double> u;                // [n_tau nq][nq] left singular vectors (columns), row b nq + a
  std::vector<double> v;                // [nq][nq] right singular vectors (columns)
  int n_tau() const { return taus.empty() ? 1 : static_cast<int>(taus.size()); }
  double ctf(int b, double y) const;    // C_b(y); 1 without CTF
  double sqrt_rho(double y) const;      // sqrt(rho(y)); 1 without a spectral weight
  // Sigma_eta V_eta(y) by the Nystrom extension (the weight's sqrt(rho) cancels):
  //   sum_{b, a} sqrt(wx_a / n_tau) J_l(x_a y) C_b(y) u[b nq + a][eta]
  double G(int eta, double y) const;
  // U_eta(x, b) by the Nystrom extension:
  //   (1/Sigma_eta) sum_c sqrt(wy_c) J_l(x y_c) C_b(y_c) sqrt(rho(y_c)) v[c][eta]
  double U(int eta, double x, int b = 0) const;
};

ModalSVD modal_svd(int l, double W, int nq, const std::vector<double>& taus = {}, double phase = 0.0,
                   double decay = 0.0);

double bessel_j(int l, double x);

}  // namespace ftk
