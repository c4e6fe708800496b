// FP64 Krylov kernels and the GMRES solver (Sec. V, stage v).
//
// Vectors are complex FP64 [n][R] (R right-hand sides innermost).  The R
// systems advance in lockstep: one R-column product per Arnoldi step, classical
// Gram-Schmidt with a second pass whenever a column's norm falls below 1/sqrt(2)
// of its value before projection, Givens rotations and the small least-squares
// problems on the host in FP64.  One device->host copy per step (two when the
// second pass runs) carries the Hessenberg column of every right-hand side.
#include <chrono>
#include <cmath>

#include "smr_internal.h"

namespace smr {

// partial[j][chunk][r] = sum over rows in chunk of conj(V_j[i][r]) w[i][r]
__global__ void k_multidot_part(int J, long long n, int R, int rl, int nchunk, long long rows_per,
                                const double2* __restrict__ V, long long ldv,
                                const double2* __restrict__ w, double2* __restrict__ part) {
  int j = blockIdx.y, chunk = blockIdx.x;
  int a = threadIdx.x / R, r = threadIdx.x % R;
  double2 acc = make_double2(0, 0);
  if (a < rl) {
    const double2* v = V + (size_t)j * ldv;
    long long i0 = chunk * rows_per, i1 = min(n, i0 + rows_per);
    for (long long i = i0 + a; i < i1; i += rl) {
      double2 x = v[i * R + r], y = w[i * R + r];
      acc.x += x.x * y.x + x.y * y.y;
      acc.y += x.x * y.y - x.y * y.x;
    }
  }
  __shared__ double2 red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  if (a == 0 && r < R) {
    double2 s = make_double2(0, 0);
    for (int q = 0; q < rl; ++q) {
      double2 t = red[q * R + r];
      s.x += t.x;
      s.y += t.y;
    }
    part[((size_t)j * nchunk + chunk) * R + r] = s;
  }
}

__global__ void k_multidot_final(int J, int R, int nchunk, const double2* __restrict__ part,
                                 double2* __restrict__ h) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J * R) return;
  int j = t / R, r = t % R;
  double2 s = make_double2(0, 0);
  for (int c = 0; c < nchunk; ++c) {
    double2 v = part[((size_t)j * nchunk + c) * R + r];
    s.x += v.x;
    s.y += v.y;
  }
  h[t] = s;
}

// w[i][r] += sign * sum_j V_j[i][r] h[j][r]
__global__ void k_multi_axpy(int J, long long n, int R, const double2* __restrict__ V, long long ldv,
                             const double2* __restrict__ h, double2* __restrict__ w, double sign) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  int r = (int)(t % R);
  double2 acc = make_double2(0, 0), acc2 = make_double2(0, 0);
  int j = 0;
  for (; j + 4 <= J; j += 4) {
    double2 v0 = V[(size_t)j * ldv + t], v1 = V[(size_t)(j + 1) * ldv + t];
    double2 v2 = V[(size_t)(j + 2) * ldv + t], v3 = V[(size_t)(j + 3) * ldv + t];
    double2 c0 = h[(size_t)j * R + r], c1 = h[(size_t)(j + 1) * R + r];
    double2 c2 = h[(size_t)(j + 2) * R + r], c3 = h[(size_t)(j + 3) * R + r];
    acc.x += v0.x * c0.x - v0.y * c0.y + v1.x * c1.x - v1.y * c1.y;
    acc.y += v0.x * c0.y + v0.y * c0.x + v1.x * c1.y + v1.y * c1.x;
    acc2.x += v2.x * c2.x - v2.y * c2.y + v3.x * c3.x - v3.y * c3.y;
    acc2.y += v2.x * c2.y + v2.y * c2.x + v3.x * c3.y + v3.y * c3.x;
  }
  for (; j < J; ++j) {
    double2 v = V[(size_t)j * ldv + t], c = h[(size_t)j * R + r];
    acc.x += v.x * c.x - v.y * c.y;
    acc.y += v.x * c.y + v.y * c.x;
  }
  acc.x += acc2.x;
  acc.y += acc2.y;
  double2 o = w[t];
  o.x += sign * acc.x;
  o.y += sign * acc.y;
  w[t] = o;
}

// y = a[r] x + b[r] y
__global__ void k_axpby(long long n, int R, const double2* __restrict__ a, const double2* __restrict__ x,
                        const double2* __restrict__ b, double2* __restrict__ y) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  int r = (int)(t % R);
  double2 xa = x[t], yb = y[t], ca = a[r], cb = b[r];
  y[t] = make_double2(ca.x * xa.x - ca.y * xa.y + cb.x * yb.x - cb.y * yb.y,
                      ca.x * xa.y + ca.y * xa.x + cb.x * yb.y + cb.y * yb.x);
}

static void chunking(long long n, int R, int* rl, int* nchunk, long long* rows_per) {
  *rl = std::max(1, 256 / R);
  long long per = std::max<long long>(1024, (n + 511) / 512);
  *rows_per = per;
  *nchunk = (int)((n + per - 1) / per);
}

static int red_buffer(Ctx* c, size_t bytes) {
  if (c->red_bytes >= bytes) return SMR_OK;
  if (c->d_red) cudaFree(c->d_red);
  if (c->h_red) cudaFreeHost(c->h_red);
  c->d_red = nullptr;
  c->h_red = nullptr;
  SMR_CUDA(c, cudaMalloc((void**)&c->d_red, bytes));
  SMR_CUDA(c, cudaMallocHost((void**)&c->h_red, bytes));
  c->red_bytes = bytes;
  return SMR_OK;
}

// d_h[J][R] on the device; optional host copy.
static int multidot_dev(Ctx* c, int J, long long n, int R, const double2* V, long long ldv,
                        const double2* w, double2* d_h, double2* d_part, cudaStream_t st) {
  int rl, nchunk;
  long long per;
  chunking(n, R, &rl, &nchunk, &per);
  dim3 g(nchunk, J);
  k_multidot_part<<<g, 256, 0, st>>>(J, n, R, rl, nchunk, per, V, ldv, w, d_part);
  SMR_LAUNCH(c);
  k_multidot_final<<<(J * R + 127) / 128, 128, 0, st>>>(J, R, nchunk, d_part, d_h);
  SMR_LAUNCH(c);
  return SMR_OK;
}

int multidot(Ctx* c, int J, long long n, int R, const double2* V, long long ldv, const double2* w,
             double2* h_host, cudaStream_t st) {
  int rl, nchunk;
  long long per;
  chunking(n, R, &rl, &nchunk, &per);
  size_t need = ((size_t)J * nchunk * R + (size_t)J * R) * sizeof(double2);
  int rc = red_buffer(c, need);
  if (rc) return rc;
  double2* d_part = (double2*)c->d_red;
  double2* d_h = d_part + (size_t)J * nchunk * R;
  rc = multidot_dev(c, J, n, R, V, ldv, w, d_h, d_part, st);
  if (rc) return rc;
  SMR_CUDA(c, cudaMemcpyAsync(h_host, d_h, (size_t)J * R * sizeof(double2), cudaMemcpyDeviceToHost, st));
  SMR_CUDA(c, cudaStreamSynchronize(st));
  return SMR_OK;
}

int multi_axpy(Ctx* c, int J, long long n, int R, const double2* V, long long ldv, const double2* d_h,
               double2* w, double sign, cudaStream_t st) {
  long long tot = n * R;
  k_multi_axpy<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(J, n, R, V, ldv, d_h, w, sign);
  SMR_LAUNCH(c);
  return SMR_OK;
}

int col_norms(Ctx* c, long long n, int R, const double2* v, double* norms_host, cudaStream_t st) {
  std::vector<double2> h(R);
  int rc = multidot(c, 1, n, R, v, 0, v, h.data(), st);
  if (rc) return rc;
  for (int r = 0; r < R; ++r) norms_host[r] = std::sqrt(std::max(0.0, h[r].x));
  return SMR_OK;
}

int col_axpby(long long n, int R, const double2* d_a, const double2* x, const double2* d_b, double2* y,
              cudaStream_t st) {
  long long tot = n * R;
  k_axpby<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, R, d_a, x, d_b, y);
  return cudaGetLastError() == cudaSuccess ? SMR_OK : SMR_E_CUDA;
}

// ------------------------------------------------------------------ GMRES
namespace {

struct Work {
  double2* V = nullptr;    // [m+1][n][R]
  double2* Z = nullptr;    // [m][n][R] (flexible only)
  double2* w = nullptr;    // [n][R]
  double2* t = nullptr;    // [n][R]
  double2* coef = nullptr; // device [4][m+1][R] small coefficient area
  double2* part = nullptr; // reduction partials
};

}  // namespace

static int apply_A(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st) {
  int rc = run_near(c, R, prec, x, y, st);
  if (rc) return rc;
  return run_far(c, R, prec, x, y, true, st);
}

// Solve A d = rhs from d = d0 (in d) to per-column relative residual tol_col[r]
// (relative to ||rhs_r||) with right preconditioning; A and the
// preconditioner in precision `prec`.  Returns iterations used in *its.
static int gmres_core(Ctx* c, int R, int prec, int precond, const double2* rhs, double2* d,
                      bool have_d0, const std::vector<double>& tol_col, int maxit, int restart,
                      Work& W, int* its, int* nmv, int* n_reorth, std::vector<double>& rel_out,
                      cudaStream_t st) {
  long long n = 2LL * c->npsi * c->p;
  long long ld = n * R;
  int m = restart;
  std::vector<double> bn(R), beta(R);
  int rc = col_norms(c, n, R, rhs, bn.data(), st);
  if (rc) return rc;
  for (int r = 0; r < R; ++r)
    if (bn[r] == 0.0) bn[r] = 1.0;
  // r0 = rhs - A d0  (in W.V[0])
  double2* r0 = W.V;
  if (have_d0) {
    rc = apply_A(c, R, prec, d, W.w, st);
    if (rc) return rc;
    ++*nmv;
    SMR_CUDA(c, cudaMemcpyAsync(r0, rhs, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    std::vector<double2> one(R, make_double2(-1, 0)), un(R, make_double2(1, 0));
    SMR_CUDA(c, cudaMemcpyAsync(W.coef, one.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
    SMR_CUDA(c, cudaMemcpyAsync(W.coef + R, un.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
    rc = col_axpby(n, R, W.coef, W.w, W.coef + R, r0, st);
    if (rc) { c->err = "axpby launch"; return rc; }
  } else {
    SMR_CUDA(c, cudaMemcpyAsync(r0, rhs, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SMR_CUDA(c, cudaMemsetAsync(d, 0, ld * sizeof(double2), st));
  }
  std::vector<int> done(R, 0);
  rel_out.assign(R, 1.0);
  // host Hessenberg storage per column (rotated), rotations, rhs g
  std::vector<std::complex<double>> H((size_t)(m + 1) * m * R), g((size_t)(m + 1) * R);
  std::vector<std::complex<double>> cs((size_t)m * R), sn((size_t)m * R);
  std::vector<double2> hbuf((size_t)(2 * (m + 1) + 2) * R);
  while (true) {
    rc = col_norms(c, n, R, r0, beta.data(), st);
    if (rc) return rc;
    bool all = true;
    for (int r = 0; r < R; ++r) {
      rel_out[r] = beta[r] / bn[r];
      if (!std::isfinite(beta[r])) { c->err = "NaN in residual"; return SMR_E_NAN; }
      if (rel_out[r] <= tol_col[r]) done[r] = 1;
      all = all && done[r];
    }
    if (all || *its >= maxit) return all ? SMR_OK : SMR_E_NOT_CONVERGED;
    // V0 = r0 / beta
    std::vector<double2> sc(R), zr(R, make_double2(0, 0));
    for (int r = 0; r < R; ++r) sc[r] = make_double2(beta[r] > 0 ? 1.0 / beta[r] : 0.0, 0);
    SMR_CUDA(c, cudaMemcpyAsync(W.coef, sc.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
    SMR_CUDA(c, cudaMemcpyAsync(W.coef + R, zr.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
    rc = col_axpby(n, R, W.coef, r0, W.coef + R, r0, st);
    if (rc) return rc;
    std::fill(g.begin(), g.end(), std::complex<double>(0, 0));
    for (int r = 0; r < R; ++r) g[r] = beta[r];
    std::vector<int> jend(R, 0), active(R, 0);
    for (int r = 0; r < R; ++r) active[r] = !done[r];
    int j = 0;
    for (; j < m && *its < maxit; ++j) {
      double2* Vj = W.V + (size_t)j * ld;
      // z_j = M^-1 v_j in W.t (fixed address, so one captured graph serves
      // every product of the solve); the flexible variant keeps a copy in Z_j
      if (precond == SMR_PRECOND_BLOCKDIAG) {
        rc = run_precond(c, R, prec, Vj, W.t, st);
      } else {
        SMR_CUDA(c, cudaMemcpyAsync(W.t, Vj, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      }
      if (rc) return rc;
      if (W.Z)
        SMR_CUDA(c, cudaMemcpyAsync(W.Z + (size_t)j * ld, W.t, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      rc = run_matvec_graph(c, R, prec, W.t, W.w, st);
      if (rc) return rc;
      ++*nmv;
      ++*its;
      // classical Gram-Schmidt against V_0..V_j, repeated once when the norm
      // drops below 1/sqrt(2) of its value before the projection ("twice is
      // enough"); every sum in FP64
      double2* dh1 = W.coef;                       // [j+1][R]
      double2* dh2 = W.coef + (size_t)(m + 1) * R; // [j+1][R]
      double2* dnr = W.coef + (size_t)2 * (m + 1) * R;          // ||w'||^2  [R]
      double2* dn0 = W.coef + (size_t)2 * (m + 1) * R + R;      // ||w||^2   [R]
      rc = multidot_dev(c, 1, n, R, W.w, 0, W.w, dn0, W.part, st);
      if (rc) return rc;
      rc = multidot_dev(c, j + 1, n, R, W.V, ld, W.w, dh1, W.part, st);
      if (rc) return rc;
      rc = multi_axpy(c, j + 1, n, R, W.V, ld, dh1, W.w, -1.0, st);
      if (rc) return rc;
      rc = multidot_dev(c, 1, n, R, W.w, 0, W.w, dnr, W.part, st);
      if (rc) return rc;
      SMR_CUDA(c, cudaMemcpyAsync(hbuf.data(), W.coef, (size_t)(2 * (m + 1) + 2) * R * sizeof(double2),
                                  cudaMemcpyDeviceToHost, st));
      SMR_CUDA(c, cudaStreamSynchronize(st));
      bool reorth = false;
      for (int r = 0; r < R; ++r) {
        double a0 = hbuf[(size_t)2 * (m + 1) * R + R + r].x, a1 = hbuf[(size_t)2 * (m + 1) * R + r].x;
        if (active[r] && a1 < 0.5 * a0) reorth = true;
      }
      if (reorth) {
        ++*n_reorth;
        rc = multidot_dev(c, j + 1, n, R, W.V, ld, W.w, dh2, W.part, st);
        if (rc) return rc;
        rc = multi_axpy(c, j + 1, n, R, W.V, ld, dh2, W.w, -1.0, st);
        if (rc) return rc;
        rc = multidot_dev(c, 1, n, R, W.w, 0, W.w, dnr, W.part, st);
        if (rc) return rc;
        SMR_CUDA(c, cudaMemcpyAsync(hbuf.data() + (size_t)(m + 1) * R, dh2,
                                    (size_t)((m + 1) + 1) * R * sizeof(double2), cudaMemcpyDeviceToHost, st));
        SMR_CUDA(c, cudaStreamSynchronize(st));
      } else {
        for (size_t q = 0; q < (size_t)(m + 1) * R; ++q) hbuf[(size_t)(m + 1) * R + q] = make_double2(0, 0);
      }
      // next basis vector V_{j+1} = w / ||w||
      std::vector<double2> inv(R), zz(R, make_double2(0, 0));
      std::vector<double> hn(R);
      for (int r = 0; r < R; ++r) {
        hn[r] = std::sqrt(std::max(0.0, hbuf[(size_t)2 * (m + 1) * R + r].x));
        inv[r] = make_double2(hn[r] > 0 ? 1.0 / hn[r] : 0.0, 0);
      }
      double2* Vn = W.V + (size_t)(j + 1) * ld;
      SMR_CUDA(c, cudaMemcpyAsync(W.coef + (size_t)3 * (m + 1) * R, inv.data(), R * sizeof(double2),
                                  cudaMemcpyHostToDevice, st));
      SMR_CUDA(c, cudaMemcpyAsync(W.coef + (size_t)3 * (m + 1) * R + R, zz.data(), R * sizeof(double2),
                                  cudaMemcpyHostToDevice, st));
      SMR_CUDA(c, cudaMemcpyAsync(Vn, W.w, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      rc = col_axpby(n, R, W.coef + (size_t)3 * (m + 1) * R, W.w, W.coef + (size_t)3 * (m + 1) * R + R,
                     Vn, st);
      if (rc) return rc;
      bool any = false;
      for (int r = 0; r < R; ++r) {
        if (!active[r]) continue;
        std::complex<double>* Hc = &H[((size_t)r * m + j) * (m + 1)];   // column j of column-set r
        for (int i = 0; i <= j; ++i) {
          double2 a = hbuf[(size_t)i * R + r], b = hbuf[(size_t)(m + 1) * R + (size_t)i * R + r];
          Hc[i] = std::complex<double>(a.x + b.x, a.y + b.y);
        }
        Hc[j + 1] = hn[r];
        for (int i = 0; i < j; ++i) {
          std::complex<double> ci = cs[(size_t)r * m + i], si = sn[(size_t)r * m + i];
          std::complex<double> t = ci * Hc[i] + si * Hc[i + 1];
          Hc[i + 1] = -std::conj(si) * Hc[i] + ci * Hc[i + 1];
          Hc[i] = t;
        }
        std::complex<double> a = Hc[j], b = Hc[j + 1];
        double den = std::sqrt(std::norm(a) + std::norm(b));
        std::complex<double> ci, si;
        if (den == 0.0) { ci = 1.0; si = 0.0; }
        else if (std::abs(a) == 0.0) { ci = 0.0; si = std::conj(b) / std::abs(b); }
        else { ci = std::abs(a) / den; si = (a / std::abs(a)) * std::conj(b) / den; }
        cs[(size_t)r * m + j] = ci;
        sn[(size_t)r * m + j] = si;
        Hc[j] = ci * a + si * b;
        Hc[j + 1] = 0.0;
        std::complex<double>* gr = &g[(size_t)r * (m + 1)];
        gr[j + 1] = -std::conj(si) * gr[j];
        gr[j] = ci * gr[j];
        jend[r] = j + 1;
        double est = std::abs(gr[j + 1]) / bn[r];
        rel_out[r] = est;
        if (!std::isfinite(est)) { c->err = "NaN in Givens update"; return SMR_E_NAN; }
        if (est <= tol_col[r] || hn[r] == 0.0) active[r] = 0;
        any = any || active[r];
      }
      if (!any) { ++j; break; }
    }
    // y per column: back substitution; coefficients [jmax][R] on the device
    int jmax = 0;
    for (int r = 0; r < R; ++r) jmax = std::max(jmax, jend[r]);
    std::vector<double2> ycoef((size_t)std::max(jmax, 1) * R, make_double2(0, 0));
    for (int r = 0; r < R; ++r) {
      int J = jend[r];
      std::vector<std::complex<double>> y(J);
      for (int i = J - 1; i >= 0; --i) {
        std::complex<double> s = g[(size_t)r * (m + 1) + i];
        for (int q = i + 1; q < J; ++q) s -= H[((size_t)r * m + q) * (m + 1) + i] * y[q];
        std::complex<double> diag = H[((size_t)r * m + i) * (m + 1) + i];
        y[i] = (diag != 0.0) ? s / diag : 0.0;
      }
      for (int i = 0; i < J; ++i) ycoef[(size_t)i * R + r] = make_double2(y[i].real(), y[i].imag());
    }
    if (jmax > 0) {
      SMR_CUDA(c, cudaMemcpyAsync(W.coef, ycoef.data(), (size_t)jmax * R * sizeof(double2),
                                  cudaMemcpyHostToDevice, st));
      if (W.Z) {
        rc = multi_axpy(c, jmax, n, R, W.Z, ld, W.coef, d, 1.0, st);
      } else {
        SMR_CUDA(c, cudaMemsetAsync(W.w, 0, ld * sizeof(double2), st));
        rc = multi_axpy(c, jmax, n, R, W.V, ld, W.coef, W.w, 1.0, st);
        if (rc) return rc;
        if (precond == SMR_PRECOND_BLOCKDIAG) {
          rc = run_precond(c, R, prec, W.w, W.t, st);
        } else {
          SMR_CUDA(c, cudaMemcpyAsync(W.t, W.w, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        }
        if (rc) return rc;
        std::vector<double2> one(R, make_double2(1, 0));
        SMR_CUDA(c, cudaMemcpyAsync(W.coef, one.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
        rc = col_axpby(n, R, W.coef, W.t, W.coef, d, st);
      }
      if (rc) return rc;
    }
    // true residual of this operator: r0 = rhs - A d
    rc = apply_A(c, R, prec, d, W.w, st);
    if (rc) return rc;
    ++*nmv;
    SMR_CUDA(c, cudaMemcpyAsync(r0, rhs, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    std::vector<double2> mone(R, make_double2(-1, 0)), one(R, make_double2(1, 0));
    SMR_CUDA(c, cudaMemcpyAsync(W.coef, mone.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
    SMR_CUDA(c, cudaMemcpyAsync(W.coef + R, one.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
    rc = col_axpby(n, R, W.coef, W.w, W.coef + R, r0, st);
    if (rc) return rc;
  }
}

int solve(Ctx* c, int R, const double2* b, double2* x, const smr_solve_opts* o, smr_solve_stats* stats,
          cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  long long n = 2LL * c->npsi * c->p;
  long long ld = n * R;
  int maxit = o->maxit > 0 ? o->maxit : 2000;
  int m = (o->restart > 0) ? std::min(o->restart, maxit) : maxit;
  // cap the Krylov dimension by device memory (60% of what is free)
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  bool flex = (o->precision == SMR_PREC_FP32);
  double per = (double)ld * sizeof(double2) * (flex ? 2.0 : 1.0);
  int mcap = (int)std::max(2.0, 0.6 * (double)freeb / per - 4);
  m = std::max(1, std::min(m, mcap));
  Work W;
  size_t vbytes = (size_t)(m + 1) * ld * sizeof(double2);
  SMR_CUDA(c, cudaMalloc((void**)&W.V, vbytes));
  if (flex) SMR_CUDA(c, cudaMalloc((void**)&W.Z, (size_t)m * ld * sizeof(double2)));
  SMR_CUDA(c, cudaMalloc((void**)&W.w, ld * sizeof(double2)));
  SMR_CUDA(c, cudaMalloc((void**)&W.t, ld * sizeof(double2)));
  SMR_CUDA(c, cudaMalloc((void**)&W.coef, (size_t)4 * (m + 2) * R * sizeof(double2)));
  int rl, nchunk;
  long long rows;
  chunking(n, R, &rl, &nchunk, &rows);
  SMR_CUDA(c, cudaMalloc((void**)&W.part, (size_t)(m + 2) * nchunk * R * sizeof(double2)));
  auto cleanup = [&]() {
    cudaFree(W.V); cudaFree(W.Z); cudaFree(W.w); cudaFree(W.t); cudaFree(W.coef); cudaFree(W.part);
  };
  int its = 0, mv64 = 0, mv32 = 0, outer = 0, nreo = 0, rc = SMR_OK;
  std::vector<double> rel;
  double tol = o->tol > 0 ? o->tol : 1e-4;
  if (o->precision == SMR_PREC_FP64) {
    std::vector<double> tc(R, tol);
    rc = gmres_core(c, R, SMR_PREC_FP64, o->precond, b, x, o->use_x0 != 0, tc, maxit, m, W, &its,
                    &mv64, &nreo, rel, st);
  } else {
    // iterative refinement: outer FP64 residual, inner FGMRES on the FP32 product
    double2 *r = nullptr, *dlt = nullptr;
    SMR_CUDA(c, cudaMalloc((void**)&r, ld * sizeof(double2)));
    SMR_CUDA(c, cudaMalloc((void**)&dlt, ld * sizeof(double2)));
    std::vector<double> bn(R), rn(R);
    rc = col_norms(c, n, R, b, bn.data(), st);
    if (!o->use_x0) SMR_CUDA(c, cudaMemsetAsync(x, 0, ld * sizeof(double2), st));
    int max_outer = o->max_outer > 0 ? o->max_outer : 8;
    while (rc == SMR_OK) {
      // r = b - A64 x
      if (outer == 0 && !o->use_x0) {
        SMR_CUDA(c, cudaMemcpyAsync(r, b, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      } else {
        rc = apply_A(c, R, SMR_PREC_FP64, x, W.w, st);
        if (rc) break;
        ++mv64;
        SMR_CUDA(c, cudaMemcpyAsync(r, b, ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        std::vector<double2> mone(R, make_double2(-1, 0)), one(R, make_double2(1, 0));
        SMR_CUDA(c, cudaMemcpyAsync(W.coef, mone.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
        SMR_CUDA(c, cudaMemcpyAsync(W.coef + R, one.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
        rc = col_axpby(n, R, W.coef, W.w, W.coef + R, r, st);
        if (rc) break;
      }
      rc = col_norms(c, n, R, r, rn.data(), st);
      if (rc) break;
      bool all = true;
      std::vector<double> tc(R);
      rel.assign(R, 0.0);
      for (int q = 0; q < R; ++q) {
        double bq = bn[q] > 0 ? bn[q] : 1.0;
        rel[q] = rn[q] / bq;
        all = all && rel[q] <= tol;
        // inner target: leave half the budget for the FP32 product error
        tc[q] = (rn[q] > 0) ? std::max(0.5 * tol * bq / rn[q], 1e-7) : 1.0;
      }
      if (all) break;
      if (outer >= max_outer || its >= maxit) { rc = SMR_E_NOT_CONVERGED; break; }
      std::vector<double> rel_in;
      int rci = gmres_core(c, R, SMR_PREC_FP32, o->precond, r, dlt, false, tc, maxit - its, m, W,
                           &its, &mv32, &nreo, rel_in, st);
      if (rci && rci != SMR_E_NOT_CONVERGED) { rc = rci; break; }
      std::vector<double2> one(R, make_double2(1, 0));
      SMR_CUDA(c, cudaMemcpyAsync(W.coef, one.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st));
      rc = col_axpby(n, R, W.coef, dlt, W.coef, x, st);
      ++outer;
    }
    cudaFree(r);
    cudaFree(dlt);
  }
  SMR_CUDA(c, cudaStreamSynchronize(st));
  cleanup();
  if (stats) {
    stats->iters = its;
    stats->matvecs_fp64 = mv64;
    stats->matvecs_fp32 = mv32;
    stats->outer = outer;
    stats->reorth = nreo;
    double mx = 0;
    for (double v : rel) mx = std::max(mx, v);
    stats->resid_true = mx;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

}  // namespace smr
