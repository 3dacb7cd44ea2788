// Plan-time eigen-data of the 1D absorbing pencil (K, M), host FP64.
//
// The solver's Step 2 (Section 4.2.2, eqs. step2-1..step2-3) needs, per x1 mode
// l, the eigenvalue Lam^A_l of K V = M V Lam^A (eq. EVP1a) and the boundary
// rows V[1,l], V[n,l] of the eigenvectors normalised by V^T M V = I (eq.
// EVPcondA).  The paper obtains them from a dense eigensolver during its
// initialisation.  Here they come from an O(n^2) method that uses the
// structure of the pencil:
//
//   K = K^N - i w (e_1 e_1^T + e_n e_n^T),
//
// where K^N is the Neumann stiffness (k11 = knn = 1, eq. matrixK).  The
// Neumann pencil (K^N, M) is diagonalised by cosines phi_k(j) = c_k cos(k pi
// (j-1)/(n-1)), k = 0..n-1, with eigenvalues kappa_k/mu_k, kappa_k =
// (2 - 2 cos t_k)/h, and M-normalisation weights w_k = phi_k(1)^2 =
// 2/(mu_k (n-1)) (halved for k = 0 and k = n-1), mu_k = h ((den - 2) +
// 2 cos t_k)/den for the mass h [(den-2)/den, 1/den] with half-weight ends
// (den = 6: eq. matrixM, mu_k = h (2 + cos t_k)/3; den = 12: the modified
// elements).  The pencil is symmetric under
// j -> n+1-j, so eigenvectors are even (v_1 = v_n, only even k) or odd
// (v_n = -v_1, only odd k), and each eigenvalue solves the secular equation
//
//   F(lam) = 1 - 2 i w sum_{k in class} w_k / (lam_k - lam) = 0.
//
// With v_1 = 1 the eigenvector is v = sum_k a_k phi_k, a_k = 2 i w phi_k(1) /
// (lam_k - lam), so v^T M v = -4 w^2 S2, S2 = sum_k w_k/(lam_k - lam)^2, and
// the normalised boundary entries satisfy V[1,l]^2 = -1/(4 w^2 S2) and
// V[n,l] = +-V[1,l].  Step 2 only ever uses V[1,l]^2 and V[1,l] V[n,l], so
// (lam, sigma = V[1,l]^2, parity) is all the solver stores.
//
// All roots of each class are found together by the Aberth-Ehrlich iteration
// on the polynomial F(lam) prod_k (lam_k - lam), started from the first-order
// perturbation lam_k - 2 i w w_k, then polished by Newton steps on F.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <thread>
#include <vector>

#include "helm_internal.h"

namespace helm {

namespace {

struct cd {
  double re, im;
};
inline cd cadd(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
inline cd csub(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
inline cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cd crecip(cd a) {
  // Smith-style scaling keeps the reciprocal accurate for any magnitude.
  if (std::fabs(a.re) >= std::fabs(a.im)) {
    double r = a.im / a.re, d = a.re + a.im * r;
    return {1.0 / d, -r / d};
  }
  double r = a.re / a.im, d = a.re * r + a.im;
  return {r / d, -1.0 / d};
}
inline cd cdiv(cd a, cd b) { return cmul(a, crecip(b)); }
inline double cabs_(cd a) { return std::hypot(a.re, a.im); }

template <typename Fn>
void parallel_for(int64_t n, Fn fn) {
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int64_t nt = std::min<int64_t>(hw, std::max<int64_t>(1, n / 64));
  if (nt <= 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a < b) th.emplace_back([=] { fn(a, b); });
  }
  for (auto& x : th) x.join();
}

// One symmetry class: poles lk, weights wk (size m).  Returns roots and S2.
int solve_class(const std::vector<double>& lk, const std::vector<double>& wk, double omega,
                std::vector<cd>& z, std::vector<cd>& s2) {
  const int64_t m = (int64_t)lk.size();
  z.resize(m);
  s2.resize(m);
  const cd tiw = {0.0, 2.0 * omega};  // 2 i w
  for (int64_t j = 0; j < m; ++j) z[j] = {lk[j], -2.0 * omega * wk[j]};
  std::vector<cd> step(m);
  std::vector<char> active(m, 1);
  const int maxit = 500;
  int it = 0;
  for (; it < maxit; ++it) {
    parallel_for(m, [&](int64_t a, int64_t b) {
      for (int64_t j = a; j < b; ++j) {
        if (!active[j]) {
          step[j] = {0, 0};
          continue;
        }
        cd zj = z[j];
        cd sF = {0, 0}, sF2 = {0, 0}, sQ = {0, 0}, sA = {0, 0};
        for (int64_t k = 0; k < m; ++k) {
          cd d = {lk[k] - zj.re, -zj.im};  // lam_k - z
          cd r = crecip(d);
          cd wr = {wk[k] * r.re, wk[k] * r.im};
          sF = cadd(sF, wr);
          sF2 = cadd(sF2, cmul(wr, r));
          sQ = csub(sQ, r);  // 1/(z - lam_k)
          if (k != j) sA = cadd(sA, crecip(csub(zj, z[k])));
        }
        cd F = csub({1.0, 0.0}, cmul(tiw, sF));
        cd Fp = {0, 0};
        Fp = csub(Fp, cmul(tiw, sF2));
        // p'/p = F'/F + sum 1/(z - lam_k);  N = p/p' = F / (F' + F sQ)
        cd den = cadd(Fp, cmul(F, sQ));
        if (den.re == 0.0 && den.im == 0.0) {
          step[j] = {0, 0};
          continue;
        }
        cd N = cdiv(F, den);
        cd q = csub({1.0, 0.0}, cmul(N, sA));
        step[j] = (q.re == 0.0 && q.im == 0.0) ? N : cdiv(N, q);
      }
    });
    bool any = false;
    for (int64_t j = 0; j < m; ++j) {
      if (!active[j]) continue;
      z[j] = csub(z[j], step[j]);
      if (cabs_(step[j]) <= 1e-15 * std::max(1.0, cabs_(z[j])))
        active[j] = 0;
      else
        any = true;
      if (!std::isfinite(z[j].re) || !std::isfinite(z[j].im)) return -1;
    }
    if (!any) break;
  }
  if (it == maxit) return -2;
  // Newton polish on F and the normalisation sum S2.
  parallel_for(m, [&](int64_t a, int64_t b) {
    for (int64_t j = a; j < b; ++j) {
      for (int pass = 0; pass < 3; ++pass) {
        cd zj = z[j];
        cd sF = {0, 0}, sF2 = {0, 0};
        for (int64_t k = 0; k < m; ++k) {
          cd r = crecip({lk[k] - zj.re, -zj.im});
          cd wr = {wk[k] * r.re, wk[k] * r.im};
          sF = cadd(sF, wr);
          sF2 = cadd(sF2, cmul(wr, r));
        }
        if (pass == 2) {
          s2[j] = sF2;
          break;
        }
        cd F = csub({1.0, 0.0}, cmul(tiw, sF));
        cd Fp = {0.0, 0.0};
        Fp = csub(Fp, cmul(tiw, sF2));
        if (Fp.re != 0.0 || Fp.im != 0.0) z[j] = csub(z[j], cdiv(F, Fp));
      }
    }
  });
  return 0;
}

}  // namespace

int abc_eigen(int64_t n, double h, double omega, double* lam, double* sigma, int8_t* parity, double mden) {
  if (n < 2 || !(h > 0) || !(omega >= 0) || !std::isfinite(h) || !std::isfinite(omega) || !(mden > 2.0))
    return HELM_EINVAL;
  const double pi = 3.14159265358979323846;
  std::vector<double> lamN(n), w(n);
  for (int64_t k = 0; k < n; ++k) {
    double c = std::cos(pi * (double)k / (double)(n - 1));
    // 1 - cos t computed as 2 sin^2(t/2) to keep small eigenvalues accurate
    double s = std::sin(0.5 * pi * (double)k / (double)(n - 1));
    // cosine eigenvalues of the Neumann pencil: kappa/mu with kappa =
    // (2 - 2 cos t)/h and mu = h ((den - 2) + 2 cos t)/den (the paper's
    // elements: den = 6, mu = h (2 + cos t)/3)
    double mu = mden == 6.0 ? h * (2.0 + c) / 3.0 : h * ((mden - 2.0) + 2.0 * c) / mden;
    lamN[k] = mden == 6.0 ? 6.0 / (h * h) * (2.0 * s * s) / (2.0 + c) : (4.0 * s * s / h) / mu;
    w[k] = 2.0 / (mu * (double)(n - 1));
    if (k == 0 || k == n - 1) w[k] *= 0.5;
  }
  if (omega == 0.0) {
    // w = 0: the Neumann pencil itself (corner k11 = 1 of eq. matrixK, a
    // Gamma_N axis); its eigenvectors are the cosines, V[1,k]^2 = w_k and
    // V[n,k] = (-1)^k V[1,k]
    for (int64_t k = 0; k < n; ++k) {
      lam[2 * k] = lamN[k];
      lam[2 * k + 1] = 0.0;
      sigma[2 * k] = w[k];
      sigma[2 * k + 1] = 0.0;
      parity[k] = (k & 1) ? -1 : 1;
    }
    return HELM_OK;
  }
  int64_t pos = 0;
  for (int cls = 0; cls < 2; ++cls) {
    std::vector<double> lk, wk;
    for (int64_t k = cls; k < n; k += 2) {
      lk.push_back(lamN[k]);
      wk.push_back(w[k]);
    }
    if (lk.empty()) continue;
    std::vector<cd> z, s2;
    int rc = solve_class(lk, wk, omega, z, s2);
    if (rc != 0) return HELM_ENUMERIC;
    for (size_t j = 0; j < z.size(); ++j, ++pos) {
      lam[2 * pos] = z[j].re;
      lam[2 * pos + 1] = z[j].im;
      // sigma = -1 / (4 w^2 S2)
      cd sg = crecip({-4.0 * omega * omega * s2[j].re, -4.0 * omega * omega * s2[j].im});
      if (!std::isfinite(sg.re) || !std::isfinite(sg.im)) return HELM_ENUMERIC;
      sigma[2 * pos] = sg.re;
      sigma[2 * pos + 1] = sg.im;
      parity[pos] = cls == 0 ? 1 : -1;
    }
  }
  return HELM_OK;
}

// Same eigen-data as abc_eigen, computed single-threaded in a caller-provided
// workspace of at least 8 n + 64 doubles (no heap use).  Used by the
// allocation-free solve entry point.
int abc_eigen_static(int64_t n, double h, double omega, double* lam, double* sigma, int8_t* parity, double* work,
                     int64_t work_len) {
  if (n < 2 || !(h > 0) || !(omega > 0) || !std::isfinite(h) || !std::isfinite(omega)) return HELM_EINVAL;
  const int64_t m_max = (n + 1) / 2;
  if (!work || work_len < 2 * n + 9 * m_max + 16) return HELM_EINVAL;
  const double pi = 3.14159265358979323846;
  double* lamN = work;
  double* wgt = lamN + n;
  double* lk = wgt + n;
  double* wk = lk + m_max;
  double* zr = wk + m_max;  // roots, interleaved (re, im)
  double* sr = zr + 2 * m_max;  // S2, interleaved
  double* st = sr + 2 * m_max;  // steps, interleaved
  double* act = st + 2 * m_max;
  for (int64_t k = 0; k < n; ++k) {
    double c = std::cos(pi * (double)k / (double)(n - 1));
    double s = std::sin(0.5 * pi * (double)k / (double)(n - 1));
    lamN[k] = 6.0 / (h * h) * (2.0 * s * s) / (2.0 + c);
    double mu = h * (2.0 + c) / 3.0;
    wgt[k] = 2.0 / (mu * (double)(n - 1));
    if (k == 0 || k == n - 1) wgt[k] *= 0.5;
  }
  const cd tiw = {0.0, 2.0 * omega};
  int64_t pos = 0;
  for (int cls = 0; cls < 2; ++cls) {
    int64_t m = 0;
    for (int64_t k = cls; k < n; k += 2, ++m) {
      lk[m] = lamN[k];
      wk[m] = wgt[k];
    }
    if (m == 0) continue;
    for (int64_t j = 0; j < m; ++j) {
      zr[2 * j] = lk[j];
      zr[2 * j + 1] = -2.0 * omega * wk[j];
      act[j] = 1.0;
    }
    int it = 0;
    const int maxit = 500;
    for (; it < maxit; ++it) {
      for (int64_t j = 0; j < m; ++j) {
        st[2 * j] = st[2 * j + 1] = 0.0;
        if (act[j] == 0.0) continue;
        const cd zj = {zr[2 * j], zr[2 * j + 1]};
        cd sF = {0, 0}, sF2 = {0, 0}, sQ = {0, 0}, sA = {0, 0};
        for (int64_t k = 0; k < m; ++k) {
          const cd r = crecip({lk[k] - zj.re, -zj.im});
          const cd wr = {wk[k] * r.re, wk[k] * r.im};
          sF = cadd(sF, wr);
          sF2 = cadd(sF2, cmul(wr, r));
          sQ = csub(sQ, r);
          if (k != j) sA = cadd(sA, crecip(csub(zj, {zr[2 * k], zr[2 * k + 1]})));
        }
        const cd F = csub({1.0, 0.0}, cmul(tiw, sF));
        const cd Fp = csub({0.0, 0.0}, cmul(tiw, sF2));
        const cd den = cadd(Fp, cmul(F, sQ));
        if (den.re == 0.0 && den.im == 0.0) continue;
        const cd N = cdiv(F, den);
        const cd q = csub({1.0, 0.0}, cmul(N, sA));
        const cd stp = (q.re == 0.0 && q.im == 0.0) ? N : cdiv(N, q);
        st[2 * j] = stp.re;
        st[2 * j + 1] = stp.im;
      }
      bool any = false;
      for (int64_t j = 0; j < m; ++j) {
        if (act[j] == 0.0) continue;
        zr[2 * j] -= st[2 * j];
        zr[2 * j + 1] -= st[2 * j + 1];
        if (!std::isfinite(zr[2 * j]) || !std::isfinite(zr[2 * j + 1])) return HELM_ENUMERIC;
        if (std::hypot(st[2 * j], st[2 * j + 1]) <= 1e-15 * std::max(1.0, std::hypot(zr[2 * j], zr[2 * j + 1])))
          act[j] = 0.0;
        else
          any = true;
      }
      if (!any) break;
    }
    if (it == maxit) return HELM_ENUMERIC;
    for (int64_t j = 0; j < m; ++j) {
      for (int pass = 0; pass < 3; ++pass) {
        const cd zj = {zr[2 * j], zr[2 * j + 1]};
        cd sF = {0, 0}, sF2 = {0, 0};
        for (int64_t k = 0; k < m; ++k) {
          const cd r = crecip({lk[k] - zj.re, -zj.im});
          const cd wr = {wk[k] * r.re, wk[k] * r.im};
          sF = cadd(sF, wr);
          sF2 = cadd(sF2, cmul(wr, r));
        }
        if (pass == 2) {
          sr[2 * j] = sF2.re;
          sr[2 * j + 1] = sF2.im;
          break;
        }
        const cd F = csub({1.0, 0.0}, cmul(tiw, sF));
        const cd Fp = csub({0.0, 0.0}, cmul(tiw, sF2));
        if (Fp.re != 0.0 || Fp.im != 0.0) {
          const cd d = cdiv(F, Fp);
          zr[2 * j] -= d.re;
          zr[2 * j + 1] -= d.im;
        }
      }
    }
    for (int64_t j = 0; j < m; ++j, ++pos) {
      lam[2 * pos] = zr[2 * j];
      lam[2 * pos + 1] = zr[2 * j + 1];
      const cd sg = crecip({-4.0 * omega * omega * sr[2 * j], -4.0 * omega * omega * sr[2 * j + 1]});
      if (!std::isfinite(sg.re) || !std::isfinite(sg.im)) return HELM_ENUMERIC;
      sigma[2 * pos] = sg.re;
      sigma[2 * pos + 1] = sg.im;
      parity[pos] = cls == 0 ? 1 : -1;
    }
  }
  return HELM_OK;
}

// Unit roots e^{-2 pi i k / n}, k = 0..n-1, from libm sin/cos after exact
// reduction of k/n to the first octant (symmetries of sin/cos).
void unit_roots(int64_t n, double* re, double* im) {
  const double pi = 3.14159265358979323846;
  for (int64_t k = 0; k < n; ++k) {
    // angle = 2 pi k / n = (pi/4) * (8k/n); reduce 8k mod 8n to octant
    int64_t q8 = 8 * k;  // in units of (pi/4)/n
    int64_t oct = q8 / n;          // 0..7
    int64_t rem = q8 - oct * n;    // angle within octant = (pi/4) rem / n
    double c, s;
    double t = (pi / 4.0) * (double)rem / (double)n;
    double tq = (pi / 4.0) * (double)(n - rem) / (double)n;  // pi/4 - t without cancellation
    double ct = std::cos(t), st = std::sin(t);
    double tc = std::cos(tq), ts = std::sin(tq);
    // cos/sin of oct*pi/4 + t
    switch (oct) {
      case 0: c = ct; s = st; break;
      case 1: c = ts; s = tc; break;            // pi/2 - (pi/4 - t)
      case 2: c = -st; s = ct; break;
      case 3: c = -tc; s = ts; break;
      case 4: c = -ct; s = -st; break;
      case 5: c = -ts; s = -tc; break;
      case 6: c = st; s = -ct; break;
      default: c = tc; s = -ts; break;
    }
    re[k] = c;
    im[k] = -s;  // e^{-i angle}
  }
}

int dft_factor(int64_t n, DftPlan* p) {
  p->n = (int)n;
  p->nstages = 0;
  p->bm = 0;
  p->bstages = 0;
  p->bw = p->btw = nullptr;
  p->bf[0] = p->bf[1] = nullptr;
  p->gw[0] = p->gw[1] = nullptr;
  p->gsc[0] = p->gsc[1] = nullptr;
  p->gscale = 0.0;
  if (n < 1) return 0;
  int64_t m = n;
  auto push = [&](int r) {
    if (p->nstages < kMaxStages) p->radix[p->nstages++] = r;
    m /= r;
  };
  while (m % 8 == 0) push(8);
  if (m % 4 == 0) push(4);
  if (m % 2 == 0) push(2);
  for (int64_t q = 3; m > 1; q += 2) {
    while (m % q == 0) push((int)q);
    if (q * q > m && m > 1) {
      push((int)m);
      break;
    }
  }
  return p->nstages;
}

}  // namespace helm
