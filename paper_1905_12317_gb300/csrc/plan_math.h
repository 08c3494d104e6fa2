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
struct ModalSVD {
  int l = 0;
  int nq = 0;
  double X = 0;
  std::vector<double> sigma;            // all singular values, descending
  std::vector<double> xq, sqwx;         // x nodes, sqrt of weights
  std::vector<double> yq, sqwy;         // y nodes, sqrt of weights
  std::vector<double> u;                // [nq][nq] left singular vectors (columns)
  std::vector<double> v;                // [nq][nq] right singular vectors (columns)
  // Sigma_eta V_eta(y) by the Nystrom extension: sum_a sqrt(wx_a) J_l(x_a y) u[a][eta]
  double G(int eta, double y) const;
  // U_eta(x) by the Nystrom extension: (1/Sigma_eta) sum_b sqrt(wy_b) J_l(x y_b) v[b][eta]
  double U(int eta, double x) const;
};

ModalSVD modal_svd(int l, double W, int nq);

double bessel_j(int l, double x);

}  // namespace ftk
