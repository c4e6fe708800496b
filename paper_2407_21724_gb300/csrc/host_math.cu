// Host-side special functions and small dense algebra for libsmr setup.
#include <cmath>

#include "smr_internal.h"

namespace smr {
namespace hm {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_n from the asymptotic guess; nodes returned in
  // descending order so that theta = acos(x) ascends.
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= n; ++l) {
        double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int l = 2; l <= n; ++l) {
      double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p1 = z; p0 = 1.0; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  if (n % 2 == 1) x[n / 2] = 0.0;  // exact middle node
}

// Associated Legendre P_l^m(cos t) without the Condon-Shortley phase.
static double plm(int l, int m, double ct, double st) {
  if (m < 0 || m > l) return 0.0;
  double pmm = 1.0, fact = 1.0;
  for (int i = 1; i <= m; ++i) {
    pmm *= fact * st;
    fact += 2.0;
  }
  if (l == m) return pmm;
  double pm1 = ct * (2 * m + 1) * pmm;
  if (l == m + 1) return pm1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pll = (ct * (2 * ll - 1) * pm1 - (ll + m - 1) * pmm) / (ll - m);
    pmm = pm1;
    pm1 = pll;
  }
  return pll;
}

void real_ylm(int l, int m, int kind, double theta, double phi, double* Y, double* Yt,
              double* Yp) {
  double ct = std::cos(theta), st = std::sin(theta);
  double ratio = 1.0;  // (l-m)!/(l+m)!
  for (int i = l - m + 1; i <= l + m; ++i) ratio /= i;
  double nlm = std::sqrt((2 * l + 1) / (4.0 * M_PI) * ratio);
  double p = plm(l, m, ct, st);
  double dp = (m == 0) ? -plm(l, 1, ct, st)
                       : 0.5 * ((l + m) * (l - m + 1) * plm(l, m - 1, ct, st) - plm(l, m + 1, ct, st));
  double ang, dang, c;
  if (m == 0) {
    ang = 1.0; dang = 0.0; c = nlm;
  } else if (kind == 0) {
    ang = std::cos(m * phi); dang = -m * std::sin(m * phi); c = std::sqrt(2.0) * nlm;
  } else {
    ang = std::sin(m * phi); dang = m * std::cos(m * phi); c = std::sqrt(2.0) * nlm;
  }
  *Y = c * p * ang;
  *Yt = c * dp * ang;
  *Yp = c * p / st * dang;
}

void sph_bessel(int L, double x, std::vector<double>& j, std::vector<double>& y) {
  j.assign(L + 1, 0.0);
  y.assign(L + 1, 0.0);
  // y_l: upward recurrence (stable)
  y[0] = -std::cos(x) / x;
  if (L >= 1) y[1] = -std::cos(x) / (x * x) - std::sin(x) / x;
  for (int l = 1; l < L; ++l) y[l + 1] = (2.0 * l + 1.0) / x * y[l] - y[l - 1];
  // j_l: Miller's downward recurrence from well above max(L, x), normalised to j_0
  int start = L + 40 + (int)x;
  std::vector<double> f(start + 2, 0.0);
  f[start + 1] = 0.0;
  f[start] = 1e-300;
  for (int l = start; l >= 1; --l) {
    f[l - 1] = (2.0 * l + 1.0) / x * f[l] - f[l + 1];
    if (std::fabs(f[l - 1]) > 1e250) {  // rescale to stay in range
      for (int q = l - 1; q <= start + 1; ++q) f[q] *= 1e-250;
    }
  }
  double j0 = std::sin(x) / x;
  double j1 = std::sin(x) / (x * x) - std::cos(x) / x;
  double scale = (std::fabs(j0) >= std::fabs(j1)) ? j0 / f[0] : j1 / f[1];
  for (int l = 0; l <= L; ++l) j[l] = f[l] * scale;
}

void riccati(int l, double x, double* psi, double* dpsi, cd* xi, cd* dxi) {
  std::vector<double> j, y;
  sph_bessel(l + 1, x, j, y);
  // derivatives: z_l' = z_{l-1} - (l+1)/x z_l  (l >= 1);  z_0' = -z_1
  double dj = (l == 0) ? -j[1] : j[l - 1] - (l + 1.0) / x * j[l];
  double dy = (l == 0) ? -y[1] : y[l - 1] - (l + 1.0) / x * y[l];
  *psi = x * j[l];
  *dpsi = j[l] + x * dj;
  cd h(j[l], -y[l]);
  cd dh(dj, -dy);
  *xi = x * h;
  *dxi = h + x * dh;
}

bool invert(int n, std::vector<cd>& a) {
  std::vector<cd> inv(n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = std::abs(a[col * n + col]);
    for (int r = col + 1; r < n; ++r)
      if (std::abs(a[r * n + col]) > best) { best = std::abs(a[r * n + col]); piv = r; }
    if (best == 0.0) return false;
    if (piv != col)
      for (int q = 0; q < n; ++q) {
        std::swap(a[piv * n + q], a[col * n + q]);
        std::swap(inv[piv * n + q], inv[col * n + q]);
      }
    cd d = 1.0 / a[col * n + col];
    for (int q = 0; q < n; ++q) { a[col * n + q] *= d; inv[col * n + q] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      cd f = a[r * n + col];
      if (f == cd(0, 0)) continue;
      for (int q = 0; q < n; ++q) {
        a[r * n + q] -= f * a[col * n + q];
        inv[r * n + q] -= f * inv[col * n + q];
      }
    }
  }
  a.swap(inv);
  return true;
}

void mode_list(int n, std::vector<int>& l, std::vector<int>& m, std::vector<int>& kind) {
  l.clear(); m.clear(); kind.clear();
  for (int ll = 1; (int)l.size() < n; ++ll) {
    // within a shell: m = 0, then (m, cos), (m, sin) for m = 1..l
    for (int q = 0; q <= 2 * ll && (int)l.size() < n; ++q) {
      int mm = (q + 1) / 2;
      int kk = (q == 0) ? 0 : ((q % 2 == 1) ? 0 : 1);
      l.push_back(ll); m.push_back(mm); kind.push_back(kk);
    }
  }
}

}  // namespace hm
}  // namespace smr
