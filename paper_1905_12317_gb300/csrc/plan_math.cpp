// Host FP64 numerics for the FTK plan (Section 3.1 radial rule, Section 4.5
// operator SVD). Own implementations: Golub--Welsch for Gauss--Jacobi rules,
// cyclic Jacobi for the symmetric eigenproblem, one-sided Jacobi for the SVD.
#include "plan_math.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace ftk {

double bessel_j(int l, double x) {
  if (l < 0) return ((-l) & 1 ? -1.0 : 1.0) * bessel_j(-l, x);
  if (x == 0.0) return l == 0 ? 1.0 : 0.0;
  return std::cyl_bessel_j(static_cast<double>(l), x);
}

void symmetric_eigen(int n, std::vector<double>& A, std::vector<double>& e, std::vector<double>& V) {
  V.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[static_cast<size_t>(i) * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[static_cast<size_t>(i) * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a(i, i) * a(i, i);
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double& vkp = V[static_cast<size_t>(k) * n + p];
          double& vkq = V[static_cast<size_t>(k) * n + q];
          const double x = vkp, y = vkq;
          vkp = c * x - s * y;
          vkq = s * x + c * y;
        }
      }
    }
  }
  e.resize(n);
  for (int i = 0; i < n; ++i) e[i] = a(i, i);
}

void gauss_jacobi(int n, double alpha, double beta, std::vector<double>& t, std::vector<double>& w) {
  // Jacobi matrix of the monic Jacobi recurrence: diagonal a_k, off-diagonal sqrt(b_k).
  std::vector<double> J(static_cast<size_t>(n) * n, 0.0);
  const double ab = alpha + beta;
  for (int k = 0; k < n; ++k) {
    const double d = 2.0 * k + ab;
    double ak;
    if (k == 0) ak = (beta - alpha) / (ab + 2.0);
    else ak = (beta * beta - alpha * alpha) / (d * (d + 2.0));
    J[static_cast<size_t>(k) * n + k] = ak;
    if (k >= 1) {
      double bk;
      if (k == 1) bk = 4.0 * (1.0 + alpha) * (1.0 + beta) / ((2.0 + ab) * (2.0 + ab) * (3.0 + ab));
      else bk = 4.0 * k * (k + alpha) * (k + beta) * (k + ab) / (d * d * (d + 1.0) * (d - 1.0));
      const double off = std::sqrt(bk);
      J[static_cast<size_t>(k) * n + (k - 1)] = off;
      J[static_cast<size_t>(k - 1) * n + k] = off;
    }
  }
  std::vector<double> e, V;
  symmetric_eigen(n, J, e, V);
  const double mu0 = std::pow(2.0, ab + 1.0) * std::tgamma(alpha + 1.0) * std::tgamma(beta + 1.0) /
                     std::tgamma(ab + 2.0);
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return e[i] < e[j]; });
  t.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    const int c = idx[i];
    t[i] = e[c];
    const double v0 = V[c];  // row 0, column c
    w[i] = mu0 * v0 * v0;
  }
}

void svd_jacobi(int m, int n, const std::vector<double>& A, std::vector<double>& U,
                std::vector<double>& s, std::vector<double>& V) {
  // Work on columns: Ac[j][i] = A[i][j].
  std::vector<double> Ac(static_cast<size_t>(n) * m), Vc(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) Ac[static_cast<size_t>(j) * m + i] = A[static_cast<size_t>(i) * n + j];
  for (int j = 0; j < n; ++j) Vc[static_cast<size_t>(j) * n + j] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n; ++p) {
      double* ap = &Ac[static_cast<size_t>(p) * m];
      for (int q = p + 1; q < n; ++q) {
        double* aq = &Ac[static_cast<size_t>(q) * m];
        double al = 0, be = 0, ga = 0;
        for (int i = 0; i < m; ++i) {
          al += ap[i] * ap[i];
          be += aq[i] * aq[i];
          ga += ap[i] * aq[i];
        }
        if (std::fabs(ga) <= 1e-15 * std::sqrt(al * be) || ga == 0.0) continue;
        rotated = true;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < m; ++i) {
          const double x = ap[i], y = aq[i];
          ap[i] = c * x - sn * y;
          aq[i] = sn * x + c * y;
        }
        double* vp = &Vc[static_cast<size_t>(p) * n];
        double* vq = &Vc[static_cast<size_t>(q) * n];
        for (int i = 0; i < n; ++i) {
          const double x = vp[i], y = vq[i];
          vp[i] = c * x - sn * y;
          vq[i] = sn * x + c * y;
        }
      }
    }
    if (!rotated) break;
  }
  std::vector<double> nrm(n);
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int i = 0; i < m; ++i) acc += Ac[static_cast<size_t>(j) * m + i] * Ac[static_cast<size_t>(j) * m + i];
    nrm[j] = std::sqrt(acc);
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
  s.resize(n);
  U.assign(static_cast<size_t>(m) * n, 0.0);
  V.assign(static_cast<size_t>(n) * n, 0.0);
  for (int k = 0; k < n; ++k) {
    const int j = idx[k];
    s[k] = nrm[j];
    const double inv = nrm[j] > 0 ? 1.0 / nrm[j] : 0.0;
    for (int i = 0; i < m; ++i) U[static_cast<size_t>(i) * n + k] = Ac[static_cast<size_t>(j) * m + i] * inv;
    for (int i = 0; i < n; ++i) V[static_cast<size_t>(i) * n + k] = Vc[static_cast<size_t>(j) * n + i];
  }
}

ModalSVD modal_svd(int l, double W, int nq, const std::vector<double>& taus, double phase, double decay) {
  ModalSVD r;
  r.l = l;
  r.nq = nq;
  r.X = 2.0 * M_PI * W;
  r.taus = taus;
  r.phase = phase;
  r.decay = decay;
  std::vector<double> t, v;
  gauss_jacobi(nq, 0.0, 1.0, t, v);
  r.xq.resize(nq);
  r.sqwx.resize(nq);
  r.yq.resize(nq);
  r.sqwy.resize(nq);
  for (int i = 0; i < nq; ++i) {
    r.xq[i] = 0.5 * r.X * (1.0 + t[i]);
    r.sqwx[i] = std::sqrt(0.25 * r.X * r.X * v[i]);
    r.yq[i] = 0.5 * (1.0 + t[i]);
    r.sqwy[i] = std::sqrt(0.25 * v[i]);
  }
  const int nt = r.n_tau();
  const double rs = 1.0 / std::sqrt(static_cast<double>(nt));
  std::vector<double> A(static_cast<size_t>(nt) * nq * nq);
  for (int b = 0; b < nt; ++b)
    for (int a = 0; a < nq; ++a)
      for (int c = 0; c < nq; ++c)
        A[(static_cast<size_t>(b) * nq + a) * nq + c] =
            rs * r.sqwx[a] * bessel_j(l, r.xq[a] * r.yq[c]) * r.ctf(b, r.yq[c]) * r.sqrt_rho(r.yq[c]) * r.sqwy[c];
  svd_jacobi(nt * nq, nq, A, r.u, r.sigma, r.v);
  return r;
}

double ModalSVD::ctf(int b, double y) const {
  return taus.empty() ? 1.0 : -std::sin(M_PI * taus[b] * y * y + phase);
}

double ModalSVD::sqrt_rho(double y) const {
  if (decay == 0.0) return 1.0;
  return std::sqrt(std::exp(-decay * y * y) * decay / -std::expm1(-decay));
}

double ModalSVD::G(int eta, double y) const {
  const int nt = n_tau();
  const double rs = 1.0 / std::sqrt(static_cast<double>(nt));
  double acc = 0.0;
  for (int b = 0; b < nt; ++b) {
    double part = 0.0;
    for (int a = 0; a < nq; ++a)
      part += sqwx[a] * bessel_j(l, xq[a] * y) * u[(static_cast<size_t>(b) * nq + a) * nq + eta];
    acc += rs * ctf(b, y) * part;
  }
  return acc;
}

double ModalSVD::U(int eta, double x, int b) const {
  double acc = 0.0;
  for (int c = 0; c < nq; ++c)
    acc += sqwy[c] * bessel_j(l, x * yq[c]) * ctf(b, yq[c]) * sqrt_rho(yq[c]) * v[static_cast<size_t>(c) * nq + eta];
  return acc / sigma[eta];
}

}  // namespace ftk
