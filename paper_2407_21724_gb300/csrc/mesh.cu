// Meshed particles: static modes (Sec. III, Eqs. 21-25) on the host in FP64,
// and the PMCHWT self block (Eqs. 13-16 with the basis change of Eq. 20) on
// the GPU in FP64.
//
// RWG functions: edge e = (i, j), i < j, edges sorted; T+ is the triangle
// whose vertex cycle runs i -> j.  Triangle t, corner a carries the half
// function h[t][a] (r - v_a) of the edge opposite corner a, h = +-l/(2 A)
// (+ on T+).  On a triangle every linear combination of RWG functions is an
// affine tangential field alpha r - beta with divergence 2 alpha.
//
// Static problems (Sec. III): stars (current out of one triangle) and loops
// (n x grad of a vertex hat function) expand and test
//   A_par  = <div s, g0 div' s'>,   A_perp = <l, g0 l'>,   G = <f, f'>
// with g0 = 1/(4 pi R).  The inner integral over the source triangle is the
// closed form of the edges (Sec. IV cites Graglia 1993 for these); the outer
// one Radon's 7-point degree-5 rule.  The outer rule makes the matrices
// slightly unsymmetric; their symmetric parts are diagonalised (Cholesky of
// G, Householder tridiagonalisation, implicit QL).  Modes: the n_perp
// largest gamma_perp, then the n_par smallest gamma_par, G-orthonormal, the
// largest RWG coefficient of each positive.
//
// Self block: for each outer point q and source triangle t' the inner
// integrals S = int G, V = int (r' - r) G, U = int (r - r') F (grad' G =
// (r - r') F) are the closed forms plus the 7-point rule applied to the
// smooth remainders G - g0 and (F - 1/(4 pi R^3)).  With mode j = alpha_j r
// - beta_j on t':
//   int psi_j G dS'           = alpha_j V + (alpha_j r - beta_j) S
//   int div psi_j G dS'       = 2 alpha_j S
//   int psi_j x grad' G dS'   = (alpha_j r - beta_j) x U
// (the last because (r' - r) x (r - r') = 0), and U is 0 for t' the test
// triangle (a principal value; the integrand is a triple product of vectors
// in one plane).  Summing over t' and then over the outer points with the
// test fields gives the mode-basis A_vec, A_div and K directly.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>

#include "smr_internal.h"

namespace smr {

namespace {

const double PI = 3.14159265358979323846;
const double FOURPI = 4.0 * PI;

int fail(Ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

// Radon's 7-point rule: barycentric points and weights (sum 1)
struct Rule7 {
  double b[7][3], w[7];
  Rule7() {
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double pts[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                              {1 - 2 * a1, a1, a1}, {a1, 1 - 2 * a1, a1}, {a1, a1, 1 - 2 * a1},
                              {1 - 2 * a2, a2, a2}, {a2, 1 - 2 * a2, a2}, {a2, a2, 1 - 2 * a2}};
    const double ws[7] = {9.0 / 40, w1, w1, w1, w2, w2, w2};
    for (int i = 0; i < 7; ++i) {
      for (int d = 0; d < 3; ++d) b[i][d] = pts[i][d];
      w[i] = ws[i];
    }
  }
};
const Rule7& rule7() {
  static const Rule7 r;
  return r;
}
// 3-point rule (degree 2) that samples the mode fields for the solver
const double TRI3[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};

__constant__ double c_r7b[21];
__constant__ double c_r7w[7];

}  // namespace

// Closed forms over a flat triangle p (3 vertices, order of the outward
// normal n) at r: I0 = int 1/R, I1 = int (r' - r)/R, I2 = int (r - r')/R^3
// (normal part 0 within eps_h of the plane: the principal value in it).
// Per edge: direction s, in-plane outward normal m = s x n, ends s+- along s
// from the foot point rho, signed distance t0 = (p_i - rho) . m,
// R0^2 = t0^2 + h^2, f = ln((R+ + s+)/(R- + s-)),
// beta = atan(t0 s+/(R0^2 + |h| R+)) - atan(t0 s-/(R0^2 + |h| R-)):
//   I0 = sum (t0 f - |h| beta),  int (r' - rho)/R = 1/2 sum m (R0^2 f + s+R+ - s-R-),
//   I2 = sum m f + sign(h) n sum beta.
__host__ __device__ inline void tri_closed(const double* r, const double* p, const double* n, double eps_h,
                                           double& I0, double* I1, double* I2) {
  const double h = (r[0] - p[0]) * n[0] + (r[1] - p[1]) * n[1] + (r[2] - p[2]) * n[2];
  const double rho[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
  const double ah = fabs(h);
  double ip[3] = {0, 0, 0}, g[3] = {0, 0, 0}, bsum = 0;
  I0 = 0;
  for (int i = 0; i < 3; ++i) {
    const double* a = p + 3 * i;
    const double* b = p + 3 * ((i + 1) % 3);
    double s[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double le = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    s[0] /= le; s[1] /= le; s[2] /= le;
    const double m[3] = {s[1] * n[2] - s[2] * n[1], s[2] * n[0] - s[0] * n[2], s[0] * n[1] - s[1] * n[0]};
    const double sp = (b[0] - rho[0]) * s[0] + (b[1] - rho[1]) * s[1] + (b[2] - rho[2]) * s[2];
    const double sm = (a[0] - rho[0]) * s[0] + (a[1] - rho[1]) * s[1] + (a[2] - rho[2]) * s[2];
    const double t0 = (a[0] - rho[0]) * m[0] + (a[1] - rho[1]) * m[1] + (a[2] - rho[2]) * m[2];
    const double R02 = t0 * t0 + h * h;
    const double Rp = sqrt(sp * sp + R02), Rm = sqrt(sm * sm + R02);
    // an edge wholly behind the foot point: the equal ratio without cancellation
    const double f = sp < 0 ? log((Rm - sm) / (Rp - sp)) : log((Rp + sp) / (Rm + sm));
    const double beta = R02 > 0 ? atan2(t0 * sp, R02 + ah * Rp) - atan2(t0 * sm, R02 + ah * Rm) : 0.0;
    I0 += t0 * f - ah * beta;
    const double c = 0.5 * (R02 * f + sp * Rp - sm * Rm);
    for (int d = 0; d < 3; ++d) {
      ip[d] += c * m[d];
      g[d] += f * m[d];
    }
    bsum += beta;
  }
  const double sg = ah > eps_h ? (h > 0 ? 1.0 : -1.0) : 0.0;
  for (int d = 0; d < 3; ++d) {
    I1[d] = ip[d] - h * I0 * n[d];
    I2[d] = g[d] + sg * bsum * n[d];
  }
}

namespace {

// ---------------------------------------------------------------- topology
struct MeshGeo {
  int nv = 0, nt = 0, ne = 0;
  std::vector<double> V;              // [nv][3]
  std::vector<int> T;                 // [nt][3]
  std::vector<double> area, nrm;      // [nt], [nt][3]
  std::vector<int> ei, ej;            // edge vertices i < j
  std::vector<double> len;            // [ne]
  std::vector<int> eo;                // [nt][3] edge opposite each corner
  std::vector<double> h;              // [nt][3] half-function factor
  double eps(int t) const {           // plane tolerance of triangle t
    double m = 1.0;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) m = std::max(m, std::fabs(V[3 * T[3 * t + a] + d]));
    return 1e-12 * m;
  }
};

int build_geo(Ctx* c, int nv, const double* verts, int nt, const int* tris, MeshGeo& g) {
  g.nv = nv;
  g.nt = nt;
  g.V.assign(verts, verts + 3 * (size_t)nv);
  g.T.assign(tris, tris + 3 * (size_t)nt);
  for (double v : g.V)
    if (!std::isfinite(v)) return fail(c, SMR_E_SHAPE, "non-finite mesh vertex");
  for (int v : g.T)
    if (v < 0 || v >= nv) return fail(c, SMR_E_SHAPE, "triangle vertex index out of range");
  g.area.resize(nt);
  g.nrm.resize(3 * (size_t)nt);
  double vol = 0;
  for (int t = 0; t < nt; ++t) {
    const double* p0 = &g.V[3 * g.T[3 * t]];
    const double* p1 = &g.V[3 * g.T[3 * t + 1]];
    const double* p2 = &g.V[3 * g.T[3 * t + 2]];
    double u[3], w[3], cr[3];
    for (int d = 0; d < 3; ++d) { u[d] = p1[d] - p0[d]; w[d] = p2[d] - p0[d]; }
    cr[0] = u[1] * w[2] - u[2] * w[1];
    cr[1] = u[2] * w[0] - u[0] * w[2];
    cr[2] = u[0] * w[1] - u[1] * w[0];
    double a2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(a2 > 0)) return fail(c, SMR_E_SHAPE, "degenerate triangle");
    g.area[t] = 0.5 * a2;
    for (int d = 0; d < 3; ++d) g.nrm[3 * t + d] = cr[d] / a2;
    vol += (p0[0] * (p1[1] * p2[2] - p1[2] * p2[1]) + p0[1] * (p1[2] * p2[0] - p1[0] * p2[2]) +
            p0[2] * (p1[0] * p2[1] - p1[1] * p2[0])) / 6.0;
  }
  // directed edges -> (triangle, corner opposite)
  std::map<std::pair<int, int>, std::pair<int, int>> dir;
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      int i = g.T[3 * t + (a + 1) % 3], j = g.T[3 * t + (a + 2) % 3];
      if (i == j) return fail(c, SMR_E_SHAPE, "triangle with a repeated vertex");
      if (!dir.emplace(std::make_pair(i, j), std::make_pair(t, a)).second)
        return fail(c, SMR_E_SHAPE, "edge used twice in one direction: inconsistent orientation");
    }
  for (auto& kv : dir)
    if (!dir.count({kv.first.second, kv.first.first})) return fail(c, SMR_E_SHAPE, "open or non-manifold mesh");
  g.ne = (int)dir.size() / 2;
  if (nv - g.ne + nt != 2) return fail(c, SMR_E_SHAPE, "mesh is not a closed genus-0 surface");
  if (!(vol > 0)) return fail(c, SMR_E_SHAPE, "normals point inwards");
  g.eo.assign(3 * (size_t)nt, -1);
  g.h.assign(3 * (size_t)nt, 0.0);
  for (auto& kv : dir) {
    int i = kv.first.first, j = kv.first.second;
    if (i > j) continue;
    int e = (int)g.ei.size();
    g.ei.push_back(i);
    g.ej.push_back(j);
    double l = 0;
    for (int d = 0; d < 3; ++d) l += (g.V[3 * j + d] - g.V[3 * i + d]) * (g.V[3 * j + d] - g.V[3 * i + d]);
    l = std::sqrt(l);
    g.len.push_back(l);
    auto tp = kv.second, tm = dir[{j, i}];
    g.eo[3 * tp.first + tp.second] = e;
    g.eo[3 * tm.first + tm.second] = e;
    g.h[3 * tp.first + tp.second] = l / (2.0 * g.area[tp.first]);
    g.h[3 * tm.first + tm.second] = -l / (2.0 * g.area[tm.first]);
  }
  return SMR_OK;
}

// parallel loop over [0, n)
template <typename F> void par_for(int n, F f) {
  int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  nth = std::min(nth, std::max(1, n / 4));
  if (nth <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (int k = 0; k < nth; ++k)
    th.emplace_back([=, &f] {
      for (int i = k; i < n; i += nth) f(i);
    });
  for (auto& t : th) t.join();
}

// Static matrices: Phi[t][t'] = int_t int_t' g0 and, on half functions,
// P[(t,a)][(t',b)] = int_t int_t' f_a . f_b g0; Gram blocks of each triangle.
void static_matrices(const MeshGeo& g, std::vector<double>& Phi, std::vector<double>& P, std::vector<double>& Gh) {
  const int nt = g.nt, nh = 3 * nt;
  const Rule7& R7 = rule7();
  Phi.assign((size_t)nt * nt, 0.0);
  P.assign((size_t)nh * nh, 0.0);
  Gh.assign((size_t)nt * 9, 0.0);
  par_for(nt, [&](int t) {
    const double* pt[3] = {&g.V[3 * g.T[3 * t]], &g.V[3 * g.T[3 * t + 1]], &g.V[3 * g.T[3 * t + 2]]};
    for (int q = 0; q < 7; ++q) {
      double r[3];
      for (int d = 0; d < 3; ++d) r[d] = R7.b[q][0] * pt[0][d] + R7.b[q][1] * pt[1][d] + R7.b[q][2] * pt[2][d];
      const double w = g.area[t] * R7.w[q];
      // Gram on t (the rule is exact)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double dot = 0;
          for (int d = 0; d < 3; ++d) dot += (r[d] - pt[a][d]) * (r[d] - pt[b][d]);
          Gh[(size_t)t * 9 + a * 3 + b] += w * g.h[3 * t + a] * g.h[3 * t + b] * dot;
        }
      for (int s = 0; s < nt; ++s) {
        double tri[9];
        for (int a = 0; a < 3; ++a)
          for (int d = 0; d < 3; ++d) tri[3 * a + d] = g.V[3 * g.T[3 * s + a] + d];
        double I0, I1[3], I2[3];
        tri_closed(r, tri, &g.nrm[3 * s], g.eps(s), I0, I1, I2);
        Phi[(size_t)t * nt + s] += w * I0 / FOURPI;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            double v = 0;
            for (int d = 0; d < 3; ++d) v += (r[d] - pt[a][d]) * (I1[d] + (r[d] - tri[3 * b + d]) * I0);
            P[(size_t)(3 * t + a) * nh + 3 * s + b] += w * g.h[3 * t + a] * g.h[3 * s + b] * v / FOURPI;
          }
      }
    }
  });
}

// sparse columns: per column, (row, value)
typedef std::vector<std::vector<std::pair<int, double>>> SpCols;

// C = X^T B X for dense B (n x n, row-major) and sparse X (n x m)
std::vector<double> sandwich(const std::vector<double>& B, int n, const SpCols& X) {
  const int m = (int)X.size();
  std::vector<double> Y((size_t)n * m, 0.0);   // B X, [n][m]
  par_for(m, [&](int j) {
    for (auto& kv : X[j])
      for (int i = 0; i < n; ++i) Y[(size_t)i * m + j] += B[(size_t)i * n + kv.first] * kv.second;
  });
  std::vector<double> C((size_t)m * m, 0.0);
  par_for(m, [&](int i) {
    for (int j = 0; j < m; ++j) {
      double s = 0;
      for (auto& kv : X[i]) s += kv.second * Y[(size_t)kv.first * m + j];
      C[(size_t)i * m + j] = s;
    }
  });
  return C;
}

// Householder reduction of the symmetric a (n x n, row-major) to
// tridiagonal form: on return a holds the orthogonal Q (A = Q T Q^T), d the
// diagonal of T and e[i] = T[i][i-1] (e[0] = 0).
void tridiagonalise(int n, std::vector<double>& a, std::vector<double>& d, std::vector<double>& e) {
  d.assign(n, 0.0);
  e.assign(n, 0.0);
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  for (int i = n - 1; i > 0; --i) {
    const int l = i - 1;
    double h = 0;
    if (l > 0) {
      double scale = 0;
      for (int k = 0; k <= l; ++k) scale += std::fabs(A(i, k));
      if (scale == 0) {
        e[i] = A(i, l);
      } else {
        for (int k = 0; k <= l; ++k) {
          A(i, k) /= scale;
          h += A(i, k) * A(i, k);
        }
        double f = A(i, l);
        double gg = f >= 0 ? -std::sqrt(h) : std::sqrt(h);
        e[i] = scale * gg;
        h -= f * gg;
        A(i, l) = f - gg;                      // u, scaled, in row i
        f = 0;
        for (int j = 0; j <= l; ++j) {
          A(j, i) = A(i, j) / h;               // u / H in column i
          double s = 0;
          for (int k = 0; k <= j; ++k) s += A(j, k) * A(i, k);
          for (int k = j + 1; k <= l; ++k) s += A(k, j) * A(i, k);
          e[j] = s / h;                        // p = A u / H
          f += e[j] * A(i, j);
        }
        const double hh = f / (h + h);
        for (int j = 0; j <= l; ++j) {         // q = p - (u.p / 2H) u;  A -= q u^T + u q^T
          f = A(i, j);
          double qj = e[j] - hh * f;
          e[j] = qj;
          for (int k = 0; k <= j; ++k) A(j, k) -= f * e[k] + qj * A(i, k);
        }
      }
    } else {
      e[i] = A(i, l);
    }
    d[i] = h;
  }
  d[0] = 0;
  e[0] = 0;
  for (int i = 0; i < n; ++i) {                 // accumulate Q
    const int l = i - 1;
    if (d[i] != 0) {
      for (int j = 0; j <= l; ++j) {
        double s = 0;
        for (int k = 0; k <= l; ++k) s += A(i, k) * A(k, j);
        for (int k = 0; k <= l; ++k) A(k, j) -= s * A(k, i);
      }
    }
    d[i] = A(i, i);
    A(i, i) = 1;
    for (int j = 0; j <= l; ++j) A(j, i) = A(i, j) = 0;
  }
}

// Eigen-decomposition of the tridiagonal (d, e) by QL with implicit shifts;
// z (n x n, row-major) holds Q on entry and the eigenvectors (columns) on
// return, d the eigenvalues (unsorted).  False if an eigenvalue needs more
// than 60 sweeps.
bool tridiagonal_ql(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& z) {
  for (int i = 1; i < n; ++i) e[i - 1] = e[i];
  e[n - 1] = 0;
  for (int l = 0; l < n; ++l) {
    int iter = 0, m;
    do {
      for (m = l; m < n - 1; ++m) {
        double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-16 * dd) break;
      }
      if (m != l) {
        if (iter++ == 60) return false;
        double gq = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = std::hypot(gq, 1.0);
        gq = d[m] - d[l] + e[l] / (gq + (gq >= 0 ? r : -r));
        double s = 1, cq = 1, p = 0;
        int i;
        for (i = m - 1; i >= l; --i) {
          double f = s * e[i], b = cq * e[i];
          r = std::hypot(f, gq);
          e[i + 1] = r;
          if (r == 0) {
            d[i + 1] -= p;
            e[m] = 0;
            break;
          }
          s = f / r;
          cq = gq / r;
          gq = d[i + 1] - p;
          r = (d[i] - gq) * s + 2.0 * cq * b;
          p = s * r;
          d[i + 1] = gq + p;
          gq = cq * r - b;
          for (int k = 0; k < n; ++k) {
            double zf = z[(size_t)k * n + i + 1];
            z[(size_t)k * n + i + 1] = s * z[(size_t)k * n + i] + cq * zf;
            z[(size_t)k * n + i] = cq * z[(size_t)k * n + i] - s * zf;
          }
        }
        if (r == 0 && i >= l) continue;
        d[l] -= p;
        e[l] = gq;
        e[m] = 0;
      }
    } while (m != l);
  }
  return true;
}

// A x = gamma B x for symmetric A (its symmetric part is used) and SPD B,
// n x n: eigenvalues ascending, eigenvectors B-orthonormal in the columns of
// X ([n][n]).  False if B is not positive definite or QL fails.
bool sym_gen_eig(int n, std::vector<double> A, std::vector<double> B, std::vector<double>& gam,
                 std::vector<double>& X) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
    }
  // Cholesky B = L L^T (lower, in place)
  for (int j = 0; j < n; ++j) {
    double s = B[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= B[(size_t)j * n + k] * B[(size_t)j * n + k];
    if (!(s > 0)) return false;
    const double ljj = std::sqrt(s);
    B[(size_t)j * n + j] = ljj;
    par_for(n - j - 1, [&](int ii) {
      const int i = j + 1 + ii;
      double t = B[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= B[(size_t)i * n + k] * B[(size_t)j * n + k];
      B[(size_t)i * n + j] = t / ljj;
    });
  }
  // W = L^-1 A (columns independent), then C = L^-1 W^T
  auto lsolve_cols = [&](std::vector<double>& M) {
    par_for(n, [&](int col) {
      for (int i = 0; i < n; ++i) {
        double t = M[(size_t)i * n + col];
        for (int k = 0; k < i; ++k) t -= B[(size_t)i * n + k] * M[(size_t)k * n + col];
        M[(size_t)i * n + col] = t / B[(size_t)i * n + i];
      }
    });
  };
  lsolve_cols(A);
  std::vector<double> C((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = A[(size_t)j * n + i];
  lsolve_cols(C);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
    }
  std::vector<double> d, e;
  tridiagonalise(n, C, d, e);
  if (!tridiagonal_ql(n, d, e, C)) return false;
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
  gam.resize(n);
  X.assign((size_t)n * n, 0.0);
  // x = L^-T y for each eigenvector y
  par_for(n, [&](int jj) {
    const int j = ord[jj];
    std::vector<double> y(n);
    for (int i = 0; i < n; ++i) y[i] = C[(size_t)i * n + j];
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= B[(size_t)k * n + i] * y[k];
      y[i] = t / B[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) X[(size_t)i * n + jj] = y[i];
    gam[jj] = d[j];
  });
  return true;
}

}  // namespace

// ---------------------------------------------------------------- static modes
namespace {
// Modes depend on the shape only (Sec. III): the last solves of this process
// are kept and reused for an identical mesh and mode counts.
struct ModeCacheEntry {
  std::vector<double> V;
  std::vector<int> T;
  int n_perp, n_par;
  MeshModes mm;
};
std::mutex g_mode_mu;
std::vector<ModeCacheEntry> g_mode_cache;
const size_t MODE_CACHE_MAX = 32;
}  // namespace

static int mesh_static_modes_solve(Ctx* c, int nv, const double* verts, int nt, const int* tris, int n_perp,
                                   int n_par, MeshModes& out);

int mesh_static_modes(Ctx* c, int nv, const double* verts, int nt, const int* tris, int n_perp, int n_par,
                      MeshModes& out) {
  {
    std::lock_guard<std::mutex> lk(g_mode_mu);
    for (const ModeCacheEntry& e : g_mode_cache)
      if (e.n_perp == n_perp && e.n_par == n_par && e.V.size() == 3 * (size_t)nv && e.T.size() == 3 * (size_t)nt &&
          std::equal(e.V.begin(), e.V.end(), verts) && std::equal(e.T.begin(), e.T.end(), tris)) {
        out = e.mm;
        return SMR_OK;
      }
  }
  int rc = mesh_static_modes_solve(c, nv, verts, nt, tris, n_perp, n_par, out);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mode_mu);
  g_mode_cache.push_back({std::vector<double>(verts, verts + 3 * (size_t)nv),
                          std::vector<int>(tris, tris + 3 * (size_t)nt), n_perp, n_par, out});
  if (g_mode_cache.size() > MODE_CACHE_MAX) g_mode_cache.erase(g_mode_cache.begin());
  return SMR_OK;
}

static int mesh_static_modes_solve(Ctx* c, int nv, const double* verts, int nt, const int* tris, int n_perp,
                                   int n_par, MeshModes& out) {
  MeshGeo g;
  int rc = build_geo(c, nv, verts, nt, tris, g);
  if (rc) return rc;
  if (n_perp > nv - 1 || n_par > nt - 1)
    return fail(c, SMR_E_SHAPE, "more modes requested than the mesh has loops (nv - 1) or stars (nt - 1)");
  std::vector<double> Phi, P, Gh;
  static_matrices(g, Phi, P, Gh);
  const int nh = 3 * nt;
  // half-function Gram (block diagonal) as a dense matrix for the sandwiches
  std::vector<double> Gd((size_t)nh * nh, 0.0);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Gd[(size_t)(3 * t + a) * nh + 3 * t + b] = Gh[(size_t)t * 9 + a * 3 + b];
  // per edge, its two halves
  std::vector<int> hp(g.ne), hm(g.ne);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) (g.h[3 * t + a] > 0 ? hp : hm)[g.eo[3 * t + a]] = 3 * t + a;
  // stars: star t holds f_e with +1 if t is T+ of e, -1 if T-; on half
  // functions that is +1 on both halves... of its own edges, per the sign of
  // the RWG function there
  const int nS = nt - 1, nL = nv - 1;
  SpCols Sh(nS), Sq(nS), Lh(nL);
  std::vector<double> Lrwg;                   // [ne][nv] loop coefficients of the RWG functions
  for (int t = 0; t < nS; ++t)
    for (int a = 0; a < 3; ++a) {
      int e = g.eo[3 * t + a];
      double sg = g.h[3 * t + a] > 0 ? 1.0 : -1.0;
      Sh[t].push_back({hp[e], sg});
      Sh[t].push_back({hm[e], sg});
    }
  // star charge per triangle: sum over the star's halves on u of 2 h
  for (int t = 0; t < nS; ++t) {
    std::map<int, double> q;
    for (auto& kv : Sh[t]) q[kv.first / 3] += kv.second * 2.0 * g.h[kv.first];
    for (auto& kv : q) Sq[t].push_back(kv);
  }
  // loops: coefficient of f_e = flux density of n x grad(lambda_v) across e out of T+
  Lrwg.assign((size_t)g.ne * nv, 0.0);
  for (int t = 0; t < nt; ++t) {
    const double* n = &g.nrm[3 * t];
    for (int a = 0; a < 3; ++a) {
      if (g.h[3 * t + a] <= 0) continue;
      const int e = g.eo[3 * t + a];
      const int i = g.T[3 * t + (a + 1) % 3], j = g.T[3 * t + (a + 2) % 3];
      double s[3], m[3];
      for (int d = 0; d < 3; ++d) s[d] = (g.V[3 * j + d] - g.V[3 * i + d]) / g.len[e];
      m[0] = s[1] * n[2] - s[2] * n[1];
      m[1] = s[2] * n[0] - s[0] * n[2];
      m[2] = s[0] * n[1] - s[1] * n[0];
      for (int v : {i, j}) {
        int k = (g.T[3 * t] == v) ? 0 : (g.T[3 * t + 1] == v ? 1 : 2);
        const double* w1 = &g.V[3 * g.T[3 * t + (k + 1) % 3]];
        const double* w2 = &g.V[3 * g.T[3 * t + (k + 2) % 3]];
        double dw[3] = {w2[0] - w1[0], w2[1] - w1[1], w2[2] - w1[2]};
        double gr[3] = {(n[1] * dw[2] - n[2] * dw[1]) / (2 * g.area[t]), (n[2] * dw[0] - n[0] * dw[2]) / (2 * g.area[t]),
                        (n[0] * dw[1] - n[1] * dw[0]) / (2 * g.area[t])};
        double J[3] = {n[1] * gr[2] - n[2] * gr[1], n[2] * gr[0] - n[0] * gr[2], n[0] * gr[1] - n[1] * gr[0]};
        Lrwg[(size_t)e * nv + v] = J[0] * m[0] + J[1] * m[1] + J[2] * m[2];
      }
    }
  }
  for (int e = 0; e < g.ne; ++e)
    for (int v : {g.ei[e], g.ej[e]})
      if (v < nL) {
        double cval = Lrwg[(size_t)e * nv + v];
        Lh[v].push_back({hp[e], cval});
        Lh[v].push_back({hm[e], cval});
      }
  std::vector<double> Apar = sandwich(Phi, nt, Sq), Gpar = sandwich(Gd, nh, Sh);
  std::vector<double> Aperp = sandwich(P, nh, Lh), Gperp = sandwich(Gd, nh, Lh);
  std::vector<double> gs, Xs, gl, Xl;
  if (!sym_gen_eig(nS, Apar, Gpar, gs, Xs) || !sym_gen_eig(nL, Aperp, Gperp, gl, Xl))
    return fail(c, SMR_E_SHAPE, "static eigenproblem failed (Gram not positive definite or no convergence)");
  const int np = n_perp + n_par;
  out.ne = g.ne;
  out.M.assign((size_t)np * g.ne, 0.0);
  out.gamma.resize(np);
  for (int i = 0; i < n_perp; ++i) {          // largest gamma_perp first
    const int col = nL - 1 - i;
    out.gamma[i] = gl[col];
    for (int e = 0; e < g.ne; ++e) {
      double s = 0;
      for (int v : {g.ei[e], g.ej[e]})
        if (v < nL) s += Lrwg[(size_t)e * nv + v] * Xl[(size_t)v * nL + col];
      out.M[(size_t)i * g.ne + e] = s;
    }
  }
  // RWG coefficient of f_e in star t: +1 on T+ (t == triangle of hp), -1 on T-
  for (int i = 0; i < n_par; ++i) {
    out.gamma[n_perp + i] = gs[i];
    for (int e = 0; e < g.ne; ++e) {
      const int tp = hp[e] / 3, tm = hm[e] / 3;
      double s = 0;
      if (tp < nS) s += Xs[(size_t)tp * nS + i];
      if (tm < nS) s -= Xs[(size_t)tm * nS + i];
      out.M[(size_t)(n_perp + i) * g.ne + e] = s;
    }
  }
  for (int i = 0; i < np; ++i) {              // the largest coefficient positive
    double* row = &out.M[(size_t)i * g.ne];
    int im = 0;
    for (int e = 1; e < g.ne; ++e)
      if (std::fabs(row[e]) > std::fabs(row[im])) im = e;
    if (row[im] < 0)
      for (int e = 0; e < g.ne; ++e) row[e] = -row[e];
  }
  // per triangle and mode: alpha, beta (psi = alpha r - beta on the triangle)
  out.nt = nt;
  out.geo_V = g.V;
  out.geo_T = g.T;
  out.area = g.area;
  out.nrm = g.nrm;
  out.ab.assign((size_t)nt * np * 4, 0.0);
  for (int t = 0; t < nt; ++t)
    for (int i = 0; i < np; ++i) {
      double al = 0, be[3] = {0, 0, 0};
      for (int a = 0; a < 3; ++a) {
        double cf = out.M[(size_t)i * g.ne + g.eo[3 * t + a]] * g.h[3 * t + a];
        al += cf;
        for (int d = 0; d < 3; ++d) be[d] += cf * g.V[3 * g.T[3 * t + a] + d];
      }
      double* o = &out.ab[((size_t)t * np + i) * 4];
      o[0] = al; o[1] = be[0]; o[2] = be[1]; o[3] = be[2];
    }
  // samples for the solver: 3-point rule per triangle
  out.nq = 3 * nt;
  out.rq.assign((size_t)out.nq * 4, 0.0);
  out.modes.assign((size_t)np * out.nq * 4, 0.0);
  for (int t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      const int q = 3 * t + k;
      double r[3];
      for (int d = 0; d < 3; ++d)
        r[d] = TRI3[k][0] * g.V[3 * g.T[3 * t] + d] + TRI3[k][1] * g.V[3 * g.T[3 * t + 1] + d] +
               TRI3[k][2] * g.V[3 * g.T[3 * t + 2] + d];
      for (int d = 0; d < 3; ++d) out.rq[4 * q + d] = r[d];
      out.rq[4 * q + 3] = g.area[t] / 3.0;
      for (int i = 0; i < np; ++i) {
        const double* o = &out.ab[((size_t)t * np + i) * 4];
        double* m = &out.modes[((size_t)i * out.nq + q) * 4];
        for (int d = 0; d < 3; ++d) m[d] = o[0] * r[d] - o[1 + d];
        m[3] = 2.0 * o[0];
      }
    }
  return SMR_OK;
}

// ---------------------------------------------------------------- self block on the GPU
namespace {

__device__ inline void smooth_parts(double k, double R, double2& g1, double2& f1) {
  const double x = k * R;
  if (x < 0.01) {
    // (e^{-jx} - 1)/x and ((1 + jx) e^{-jx} - 1)/x^2 by their series
    const double x2 = x * x;
    g1 = make_double2(k * (-x / 2 + x2 * x / 24) / FOURPI, k * (-1.0 + x2 / 6 - x2 * x2 / 120) / FOURPI);
    if (R > 0) {
      const double c = k * k / (FOURPI * R);
      f1 = make_double2(c * (0.5 - x2 / 8 + x2 * x2 / 144), c * (-x / 3 + x2 * x / 30));
    } else {
      f1 = make_double2(0.0, 0.0);
    }
    return;
  }
  double sn, cs;
  sincos(x, &sn, &cs);                        // e^{-jx} = cs - j sn
  const double iR = 1.0 / (FOURPI * R);
  g1 = make_double2((cs - 1.0) * iR, -sn * iR);
  // (1 + jx)(cs - j sn) - 1 = (cs + x sn - 1) + j (x cs - sn)
  const double iR3 = iR / (R * R);
  f1 = make_double2((cs + x * sn - 1.0) * iR3, (x * cs - sn) * iR3);
}

__device__ inline double2 cmadd(double2 acc, double a, double2 b) { return make_double2(acc.x + a * b.x, acc.y + a * b.y); }

// One block per outer point q (7 per triangle): the inner integrals against
// every source triangle into shared memory, then per mode j the sums over
// the source triangles.  X[q][j][3] = sum alpha_j (V + r S) - beta_j S,
// D[q][j] = sum 2 alpha_j S, Y[q][j][3] = sum (alpha_j r - beta_j) x U.
__global__ void k_self_inner(int nt, int npsi, const double* __restrict__ Vx, const int* __restrict__ Tx,
                             const double* __restrict__ nrm, const double* __restrict__ area,
                             const double* __restrict__ ab, double kw, double2* __restrict__ X,
                             double2* __restrict__ D, double2* __restrict__ Y) {
  extern __shared__ double2 sh[];             // [nt][7]: S, V xyz, U xyz
  const int q = blockIdx.x, tq = q / 7, iq = q % 7;
  double r[3];
  {
    const int* tt = Tx + 3 * tq;
    for (int d = 0; d < 3; ++d)
      r[d] = c_r7b[3 * iq] * Vx[3 * tt[0] + d] + c_r7b[3 * iq + 1] * Vx[3 * tt[1] + d] +
             c_r7b[3 * iq + 2] * Vx[3 * tt[2] + d];
  }
  for (int s = threadIdx.x; s < nt; s += blockDim.x) {
    double p[9], em = 1.0;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) {
        p[3 * a + d] = Vx[3 * Tx[3 * s + a] + d];
        em = fmax(em, fabs(p[3 * a + d]));
      }
    double I0, I1[3], I2[3];
    tri_closed(r, p, nrm + 3 * s, 1e-12 * em, I0, I1, I2);
    double2 S = make_double2(I0 / FOURPI, 0.0);
    double2 V[3], U[3];
    for (int d = 0; d < 3; ++d) {
      V[d] = make_double2(I1[d] / FOURPI, 0.0);
      U[d] = make_double2(I2[d] / FOURPI, 0.0);
    }
    for (int i = 0; i < 7; ++i) {
      double dv[3];
      for (int d = 0; d < 3; ++d)
        dv[d] = r[d] - (c_r7b[3 * i] * p[d] + c_r7b[3 * i + 1] * p[3 + d] + c_r7b[3 * i + 2] * p[6 + d]);
      const double R = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
      double2 g1, f1;
      smooth_parts(kw, R, g1, f1);
      const double wp = area[s] * c_r7w[i];
      S = cmadd(S, wp, g1);
      for (int d = 0; d < 3; ++d) {
        V[d] = cmadd(V[d], -wp * dv[d], g1);
        U[d] = cmadd(U[d], wp * dv[d], f1);
      }
    }
    if (s == tq)
      for (int d = 0; d < 3; ++d) U[d] = make_double2(0.0, 0.0);
    double2* o = sh + (size_t)s * 7;
    o[0] = S;
    for (int d = 0; d < 3; ++d) {
      o[1 + d] = V[d];
      o[4 + d] = U[d];
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < npsi; j += blockDim.x) {
    double2 x[3], y[3], dd = make_double2(0.0, 0.0);
    for (int d = 0; d < 3; ++d) x[d] = y[d] = make_double2(0.0, 0.0);
    for (int s = 0; s < nt; ++s) {
      const double4 c = *reinterpret_cast<const double4*>(ab + ((size_t)s * npsi + j) * 4);
      const double al = c.x, be[3] = {c.y, c.z, c.w};
      const double2* o = sh + (size_t)s * 7;
      const double2 S = o[0];
      double f[3];                            // alpha r - beta: the source field extended to r
      for (int d = 0; d < 3; ++d) {
        f[d] = al * r[d] - be[d];
        x[d] = cmadd(cmadd(x[d], al, o[1 + d]), f[d], S);
      }
      dd = cmadd(dd, 2.0 * al, S);
      // f x U
      y[0] = cmadd(cmadd(y[0], f[1], o[6]), -f[2], o[5]);
      y[1] = cmadd(cmadd(y[1], f[2], o[4]), -f[0], o[6]);
      y[2] = cmadd(cmadd(y[2], f[0], o[5]), -f[1], o[4]);
    }
    const size_t b = (size_t)q * npsi + j;
    for (int d = 0; d < 3; ++d) {
      X[b * 3 + d] = x[d];
      Y[b * 3 + d] = y[d];
    }
    D[b] = dd;
  }
}

// Av[i][j] = sum_q w psi_i(q) . X_j(q), Ad[i][j] = sum_q w 2 alpha_i D_j(q),
// K[i][j] = -sum_q w psi_i(q) . Y_j(q); one thread per (i, j).
__global__ void k_self_contract(int nt, int npsi, const double* __restrict__ Vx, const int* __restrict__ Tx,
                                const double* __restrict__ area, const double* __restrict__ ab,
                                const double2* __restrict__ X, const double2* __restrict__ D,
                                const double2* __restrict__ Y, double2* __restrict__ out) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npsi * npsi) return;
  const int i = id / npsi, j = id % npsi;
  double2 av = make_double2(0, 0), ad = make_double2(0, 0), kk = make_double2(0, 0);
  for (int t = 0; t < nt; ++t) {
    const double4 c = *reinterpret_cast<const double4*>(ab + ((size_t)t * npsi + i) * 4);
    const int* tt = Tx + 3 * t;
    for (int iq = 0; iq < 7; ++iq) {
      const int q = 7 * t + iq;
      double r[3];
      for (int d = 0; d < 3; ++d)
        r[d] = c_r7b[3 * iq] * Vx[3 * tt[0] + d] + c_r7b[3 * iq + 1] * Vx[3 * tt[1] + d] +
               c_r7b[3 * iq + 2] * Vx[3 * tt[2] + d];
      const double w = area[t] * c_r7w[iq];
      const double ps[3] = {c.x * r[0] - c.y, c.x * r[1] - c.z, c.x * r[2] - c.w};
      const size_t b = (size_t)q * npsi + j;
      for (int d = 0; d < 3; ++d) {
        av = cmadd(av, w * ps[d], X[b * 3 + d]);
        kk = cmadd(kk, -w * ps[d], Y[b * 3 + d]);
      }
      ad = cmadd(ad, w * 2.0 * c.x, D[b]);
    }
  }
  out[(size_t)id * 3] = av;
  out[(size_t)id * 3 + 1] = ad;
  out[(size_t)id * 3 + 2] = kk;
}

}  // namespace

// Z_s of a meshed shape for the scene's media (Eq. 16 with delta = 1).
int mesh_self_block(Ctx* c, const Shape& sh, std::vector<cd>& Z) {
  const MeshModes& mm = sh.mm;
  const int n = sh.n_psi(), nt = mm.nt, nq7 = 7 * nt;
  const size_t smem = (size_t)nt * 7 * sizeof(double2);
  if (smem > 200 * 1024) return fail(c, SMR_E_SHAPE, "mesh too large for the self-block kernel (at most 1828 triangles)");
  {
    const Rule7& R7 = rule7();
    double b[21], w[7];
    for (int i = 0; i < 7; ++i) {
      for (int d = 0; d < 3; ++d) b[3 * i + d] = R7.b[i][d];
      w[i] = R7.w[i];
    }
    SMR_CUDA(c, cudaMemcpyToSymbol(c_r7b, b, sizeof(b)));
    SMR_CUDA(c, cudaMemcpyToSymbol(c_r7w, w, sizeof(w)));
  }
  double *dV = nullptr, *dN = nullptr, *dA = nullptr, *dAB = nullptr;
  int* dT = nullptr;
  double2 *dX = nullptr, *dD = nullptr, *dY = nullptr, *dO = nullptr;
  auto cleanup = [&]() {
    cudaFree(dV); cudaFree(dN); cudaFree(dA); cudaFree(dAB); cudaFree(dT);
    cudaFree(dX); cudaFree(dD); cudaFree(dY); cudaFree(dO);
  };
  auto up = [&](void** d, const void* h, size_t bytes) {
    return cudaMalloc(d, bytes) == cudaSuccess && cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = up((void**)&dV, mm.geo_V.data(), mm.geo_V.size() * sizeof(double)) &&
            up((void**)&dT, mm.geo_T.data(), mm.geo_T.size() * sizeof(int)) &&
            up((void**)&dN, mm.nrm.data(), mm.nrm.size() * sizeof(double)) &&
            up((void**)&dA, mm.area.data(), mm.area.size() * sizeof(double)) &&
            up((void**)&dAB, mm.ab.data(), mm.ab.size() * sizeof(double)) &&
            cudaMalloc((void**)&dX, (size_t)nq7 * n * 3 * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&dY, (size_t)nq7 * n * 3 * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&dD, (size_t)nq7 * n * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&dO, (size_t)n * n * 3 * sizeof(double2)) == cudaSuccess;
  if (!ok) {
    cleanup();
    cudaGetLastError();
    return fail(c, SMR_E_OOM, "out of device memory for a mesh self block");
  }
  if (cudaFuncSetAttribute(k_self_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
    cleanup();
    return fail(c, SMR_E_CUDA, "self-block kernel attribute");
  }
  std::vector<double2> o((size_t)n * n * 3);
  std::vector<cd> T[2], K[2];
  const double kws[2] = {c->k, c->k_in};
  for (int m = 0; m < 2; ++m) {
    k_self_inner<<<nq7, 128, smem>>>(nt, n, dV, dT, dN, dA, dAB, kws[m], dX, dD, dY);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
      k_self_contract<<<(n * n + 127) / 128, 128>>>(nt, n, dV, dT, dA, dAB, dX, dD, dY, dO);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(o.data(), dO, o.size() * sizeof(double2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cleanup();
      return fail(c, SMR_E_CUDA, std::string("mesh self block: ") + cudaGetErrorString(e));
    }
    T[m].resize((size_t)n * n);
    K[m].resize((size_t)n * n);
    const double kw = kws[m];
    for (int ij = 0; ij < n * n; ++ij) {
      cd av(o[3 * ij].x, o[3 * ij].y), ad(o[3 * ij + 1].x, o[3 * ij + 1].y);
      T[m][ij] = cd(0.0, -kw) * av + cd(0.0, 1.0 / kw) * ad;
      K[m][ij] = cd(o[3 * ij + 2].x, o[3 * ij + 2].y);
    }
  }
  cleanup();
  const int n2 = 2 * n;
  const double zo = c->zeta, zi = c->zeta_in;
  Z.assign((size_t)n2 * n2, cd(0, 0));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const size_t ij = (size_t)i * n + j;
      Z[(size_t)i * n2 + j] = zo * T[0][ij] + zi * T[1][ij];
      Z[(size_t)i * n2 + n + j] = K[0][ij] + K[1][ij];
      Z[(size_t)(n + i) * n2 + j] = -(K[0][ij] + K[1][ij]);
      Z[(size_t)(n + i) * n2 + n + j] = T[0][ij] / zo + T[1][ij] / zi;
    }
  return SMR_OK;
}

}  // namespace smr
