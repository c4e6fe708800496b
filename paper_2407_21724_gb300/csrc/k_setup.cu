// FP64 setup kernels: mode sampling, k-space patterns (Eq. 26), translation
// tables (Eq. 23), near blocks (Eq. 16), right-hand sides (Eqs. 18-19), far
// and near fields.  Everything here runs once per scene (or per output
// request) in FP64; the hot path reads FP64 or FP32 copies of these tables.
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "smr_internal.h"

namespace smr {

static const double PI = 3.14159265358979323846;

// ------------------------------------------------------------------ modes
int build_modes(Ctx* c) {
  std::vector<double> x, w;
  hm::gauss_legendre(c->opts.n_theta, x, w);
  int nt = c->opts.n_theta, np = c->opts.n_phi;
  // one point count for every shape: the sphere rule's and the largest
  // sampled shape's (shorter rules are padded with zero-weight points)
  bool any_sphere = false;
  int qmax = 0;
  for (const Shape& sh : c->shapes) {
    if (sh.sampled) qmax = std::max(qmax, sh.nq);
    else any_sphere = true;
  }
  c->Q = std::max(any_sphere ? nt * np : 0, qmax);
  const int Qs = nt * np;
  c->rule_th.resize(Qs);
  c->rule_ph.resize(Qs);
  c->rule_w1.resize(Qs);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < np; ++j) {
      int q = i * np + j;
      c->rule_th[q] = std::acos(x[i]);
      c->rule_ph[q] = 2.0 * PI * j / np;
      c->rule_w1[q] = w[i] * 2.0 * PI / np;
    }
  int S = c->S, n = c->npsi, Q = c->Q;
  std::vector<double> modes((size_t)S * n * Q * 4, 0.0), rq((size_t)S * Q * 4);
  for (int s = 0; s < S; ++s) {
    const Shape& sh = c->shapes[s];
    if (sh.sampled) {
      for (int q = 0; q < Q; ++q) {                  // padding repeats point 0 with weight 0
        const int qq = q < sh.nq ? q : 0;
        double* R = &rq[((size_t)s * Q + q) * 4];
        for (int d = 0; d < 3; ++d) R[d] = sh.rq[4 * qq + d];
        R[3] = q < sh.nq ? sh.rq[4 * qq + 3] : 0.0;
        for (int i = 0; i < n; ++i)
          for (int d = 0; d < 4; ++d)
            modes[(((size_t)s * n + i) * Q + q) * 4 + d] = q < sh.nq ? sh.modes[((size_t)i * sh.nq + q) * 4 + d] : 0.0;
      }
      continue;
    }
    double a = sh.a;
    std::vector<int> lp, mp, kp, ll, ml, kl;
    hm::mode_list(sh.n_perp, lp, mp, kp);
    hm::mode_list(sh.n_par, ll, ml, kl);
    for (int q = 0; q < Q; ++q) {
      if (q >= Qs) {                                 // padding of a longer sampled rule
        double* R = &rq[((size_t)s * Q + q) * 4];
        R[0] = a; R[1] = R[2] = R[3] = 0.0;
        continue;
      }
      double th = c->rule_th[q], ph = c->rule_ph[q];
      double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
      double rh[3] = {st * cp, st * sp, ct};
      double thh[3] = {ct * cp, ct * sp, -st};
      double phh[3] = {-sp, cp, 0.0};
      double* R = &rq[((size_t)s * Q + q) * 4];
      R[0] = a * rh[0]; R[1] = a * rh[1]; R[2] = a * rh[2];
      R[3] = a * a * c->rule_w1[q];
      for (int i = 0; i < n; ++i) {
        bool perp = i < sh.n_perp;
        int l = perp ? lp[i] : ll[i - sh.n_perp];
        int m = perp ? mp[i] : ml[i - sh.n_perp];
        int kind = perp ? kp[i] : kl[i - sh.n_perp];
        double Y, Yt, Yp;
        hm::real_ylm(l, m, kind, th, ph, &Y, &Yt, &Yp);
        double cst = 1.0 / (a * std::sqrt((double)l * (l + 1)));
        double* M = &modes[(((size_t)s * n + i) * Q + q) * 4];
        for (int d = 0; d < 3; ++d)
          M[d] = perp ? cst * (-Yp * thh[d] + Yt * phh[d]) : cst * (Yt * thh[d] + Yp * phh[d]);
        M[3] = perp ? 0.0 : -std::sqrt((double)l * (l + 1)) * Y / (a * a);
      }
    }
  }
  int rc = upload(c, &c->d_modes, modes);
  if (rc) return rc;
  return upload(c, &c->d_rq, rq);
}

__global__ void k_to32(long long n, const double2* __restrict__ a, float2* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_to32r(long long n, const double* __restrict__ a, float* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

static int copy32(Ctx* c, const double2* src, float2** dst, long long n) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (n == 0) return SMR_OK;
  SMR_CUDA(c, cudaMalloc((void**)dst, n * sizeof(float2)));
  k_to32<<<(unsigned)((n + 255) / 256), 256>>>(n, src, *dst);
  SMR_LAUNCH(c);
  return SMR_OK;
}

// ------------------------------------------------------------------ patterns (Eq. 26)
// P[s][n][comp][k] = sum_q w_q (psi_n(q) . e_comp(k)) exp(-j k khat . r_q)
__global__ void k_patterns(int S, int npsi, int Q, int K0, const double* __restrict__ modes,
                           const double* __restrict__ rq, const double* __restrict__ khat,
                           double kw, double2* __restrict__ P) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)S * npsi * K0;
  if (t >= total) return;
  int kk = (int)(t % K0);
  int n = (int)((t / K0) % npsi);
  int s = (int)(t / ((long long)K0 * npsi));
  double kx = khat[3 * kk], ky = khat[3 * kk + 1], kz = khat[3 * kk + 2];
  double st = sqrt(kx * kx + ky * ky);
  double cp = st > 0 ? kx / st : 1.0, sp = st > 0 ? ky / st : 0.0;
  double th[3] = {kz * cp, kz * sp, -st};
  double ph[3] = {-sp, cp, 0.0};
  double2 at = make_double2(0, 0), ap = make_double2(0, 0);
  const double* M = modes + ((size_t)s * npsi + n) * Q * 4;
  const double* Rr = rq + (size_t)s * Q * 4;
  for (int q = 0; q < Q; ++q) {
    const double* r = Rr + 4 * q;
    double sn, cs;
    sincos(-kw * (kx * r[0] + ky * r[1] + kz * r[2]), &sn, &cs);
    const double* m = M + 4 * q;
    double pt = r[3] * (m[0] * th[0] + m[1] * th[1] + m[2] * th[2]);
    double pp = r[3] * (m[0] * ph[0] + m[1] * ph[1] + m[2] * ph[2]);
    at.x += pt * cs; at.y += pt * sn;
    ap.x += pp * cs; ap.y += pp * sn;
  }
  P[(((size_t)s * npsi + n) * 2 + 0) * K0 + kk] = at;
  P[(((size_t)s * npsi + n) * 2 + 1) * K0 + kk] = ap;
}

int build_patterns(Ctx* c) {
  Level& L0 = c->lev[0];
  long long n = (long long)c->S * c->npsi * 2 * L0.K;
  if (c->d_P64) cudaFree(c->d_P64);
  c->d_P64 = nullptr;
  SMR_CUDA(c, cudaMalloc((void**)&c->d_P64, n * sizeof(double2)));
  long long tot = (long long)c->S * c->npsi * L0.K;
  k_patterns<<<(unsigned)((tot + 127) / 128), 128>>>(c->S, c->npsi, c->Q, L0.K, c->d_modes, c->d_rq,
                                                    L0.d_khat, c->k, c->d_P64);
  SMR_LAUNCH(c);
  return copy32(c, c->d_P64, &c->d_P32, n);
}

// ------------------------------------------------------------------ translation (Eq. 23)
// T[o][k] = -j k/(4 pi)^2 sum_l coef[o][l] P_l(khat . Xhat_o),
// coef[o][l] = (-j)^l (2l+1) h_l^(2)(k |X_o|)
__global__ void k_ttable(int noff, int K, int L, const double* __restrict__ khat,
                         const double* __restrict__ xhat, const double2* __restrict__ coef,
                         double kw, double2* __restrict__ T) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)noff * K) return;
  int kk = (int)(t % K), o = (int)(t / K);
  double x = khat[3 * kk] * xhat[3 * o] + khat[3 * kk + 1] * xhat[3 * o + 1] +
             khat[3 * kk + 2] * xhat[3 * o + 2];
  const double2* cf = coef + (size_t)o * (L + 1);
  double p0 = 1.0, p1 = x;
  double2 acc = cf[0];
  if (L >= 1) { acc.x += cf[1].x * p1; acc.y += cf[1].y * p1; }
  for (int l = 2; l <= L; ++l) {
    double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
    acc.x += cf[l].x * p2;
    acc.y += cf[l].y * p2;
    p0 = p1;
    p1 = p2;
  }
  double pre = kw / (16.0 * PI * PI);    // -j k / (4 pi)^2 = -j pre
  T[t] = make_double2(pre * acc.y, -pre * acc.x);
}

// Tables are stored for the whole 7 x 7 grid of lattice offsets, row
// (dx + 3) * 7 + (dy + 3); the 9 rows of adjacent offsets (never translated)
// are zero.
int build_translations(Ctx* c) {
  for (int s = 0; s < c->nlev; ++s) {
    Level& L = c->lev[s];
    const int noff = 49;
    if (L.d_T64) cudaFree(L.d_T64);
    L.d_T64 = nullptr;
    if (L.off_dx.empty()) continue;
    std::vector<double2> coef((size_t)noff * (L.L + 1), make_double2(0, 0));
    std::vector<double> xhat(3 * noff, 0.0);
    for (int o = 0; o < noff; ++o) {
      int dx = o / 7 - 3, dy = o % 7 - 3;
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) { xhat[3 * o] = 1.0; continue; }
      double X[2] = {dx * L.box, dy * L.box};
      double r = std::sqrt(X[0] * X[0] + X[1] * X[1]);
      xhat[3 * o] = X[0] / r; xhat[3 * o + 1] = X[1] / r; xhat[3 * o + 2] = 0.0;
      std::vector<double> jl, yl;
      hm::sph_bessel(L.L, c->k * r, jl, yl);
      cd mj(1.0, 0.0);
      for (int l = 0; l <= L.L; ++l) {
        cd h(jl[l], -yl[l]);
        cd v = mj * (double)(2 * l + 1) * h;
        coef[(size_t)o * (L.L + 1) + l] = make_double2(v.real(), v.imag());
        mj *= cd(0.0, -1.0);
      }
    }
    double2* d_coef = nullptr;
    double* d_xhat = nullptr;
    int rc = upload(c, &d_coef, coef);
    if (rc) return rc;
    rc = upload(c, &d_xhat, xhat);
    if (rc) return rc;
    SMR_CUDA(c, cudaMalloc((void**)&L.d_T64, (size_t)noff * L.K * sizeof(double2)));
    long long tot = (long long)noff * L.K;
    k_ttable<<<(unsigned)((tot + 127) / 128), 128>>>(noff, L.K, L.L, L.d_khat, d_xhat, d_coef, c->k,
                                                    L.d_T64);
    SMR_LAUNCH(c);
    SMR_CUDA(c, cudaDeviceSynchronize());
    cudaFree(d_coef);
    cudaFree(d_xhat);
    rc = copy32(c, L.d_T64, &L.d_T32, tot);
    if (rc) return rc;
  }
  return SMR_OK;
}

// ------------------------------------------------------------------ near blocks (Eq. 16)
// Stage 1: for each block (test shape sm at dc, source shape sn at 0), each test
// point q and source mode n:  F[0..2] = sum_q' w' g psi_n,   F[3] = sum w' g div_n,
// F[4..6] = sum w' gp (psi_n x d),  g = e/(4 pi R), gp = (1+jkR) e/(4 pi R^3).
__global__ void k_near_f(int nb, int npsi, int Q, const int* __restrict__ bsm,
                         const int* __restrict__ bsn, const double* __restrict__ bdc,
                         const double* __restrict__ modes, const double* __restrict__ rq,
                         double kw, double2* __restrict__ F) {
  int b = blockIdx.y;
  int n = threadIdx.x;
  int q = blockIdx.x * blockDim.y + threadIdx.y;
  if (q >= Q || n >= npsi) return;
  int sm = bsm[b], sn = bsn[b];
  const double* Pq = rq + ((size_t)sm * Q + q) * 4;
  double px = Pq[0] + bdc[3 * b], py = Pq[1] + bdc[3 * b + 1], pz = Pq[2] + bdc[3 * b + 2];
  const double* Rs = rq + (size_t)sn * Q * 4;
  const double* Ms = modes + ((size_t)sn * npsi + n) * Q * 4;
  double2 acc[7];
  for (int i = 0; i < 7; ++i) acc[i] = make_double2(0, 0);
  for (int qq = 0; qq < Q; ++qq) {
    const double* r = Rs + 4 * qq;
    double dx = px - r[0], dy = py - r[1], dz = pz - r[2];
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    double sn_, cs;
    sincos(-kw * R, &sn_, &cs);
    double iR = 1.0 / R;
    double g = r[3] * iR / (4.0 * PI);             // weight folded in
    double gr = g * cs, gi = g * sn_;               // w' g
    double g3 = g * iR * iR;
    // w' (1 + j k R) e / (4 pi R^3)
    double hr = g3 * (cs - kw * R * sn_), hi = g3 * (sn_ + kw * R * cs);
    const double* m = Ms + 4 * qq;
    acc[0].x += gr * m[0]; acc[0].y += gi * m[0];
    acc[1].x += gr * m[1]; acc[1].y += gi * m[1];
    acc[2].x += gr * m[2]; acc[2].y += gi * m[2];
    acc[3].x += gr * m[3]; acc[3].y += gi * m[3];
    double cx = m[1] * dz - m[2] * dy, cy = m[2] * dx - m[0] * dz, cz = m[0] * dy - m[1] * dx;
    acc[4].x += hr * cx; acc[4].y += hi * cx;
    acc[5].x += hr * cy; acc[5].y += hi * cy;
    acc[6].x += hr * cz; acc[6].y += hi * cz;
  }
  double2* o = F + (((size_t)b * Q + q) * npsi + n) * 7;
  for (int i = 0; i < 7; ++i) o[i] = acc[i];
}

// Stage 2: T_mn = -jk sum_q w psi_m . Fv_n + (j/k) sum_q w div_m Fd_n,
//          K_mn = - sum_q w psi_m . FK_n;  block [zT, K; -K, T/z], stored transposed.
__global__ void k_near_z(int nb, int npsi, int Q, const int* __restrict__ bsm,
                         const double* __restrict__ modes, const double* __restrict__ rq,
                         const double2* __restrict__ F, double kw, double zeta,
                         double2* __restrict__ Bt, const int* __restrict__ bidx) {
  int b = blockIdx.y;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npsi * npsi) return;
  int m = t / npsi, n = t % npsi;
  int sm = bsm[b];
  const double* Mm = modes + ((size_t)sm * npsi + m) * Q * 4;
  const double* Rm = rq + (size_t)sm * Q * 4;
  double2 v = make_double2(0, 0), d = make_double2(0, 0), kk = make_double2(0, 0);
  for (int q = 0; q < Q; ++q) {
    double w = Rm[4 * q + 3];
    const double* mm = Mm + 4 * q;
    const double2* f = F + (((size_t)b * Q + q) * npsi + n) * 7;
    v.x += w * (mm[0] * f[0].x + mm[1] * f[1].x + mm[2] * f[2].x);
    v.y += w * (mm[0] * f[0].y + mm[1] * f[1].y + mm[2] * f[2].y);
    d.x += w * mm[3] * f[3].x;
    d.y += w * mm[3] * f[3].y;
    kk.x += w * (mm[0] * f[4].x + mm[1] * f[5].x + mm[2] * f[6].x);
    kk.y += w * (mm[0] * f[4].y + mm[1] * f[5].y + mm[2] * f[6].y);
  }
  // T = -jk v + (j/k) d
  double2 T = make_double2(kw * v.y - d.y / kw, -kw * v.x + d.x / kw);
  double2 K = make_double2(-kk.x, -kk.y);
  int n2 = 2 * npsi;
  double2* B = Bt + (size_t)bidx[b] * n2 * n2;
  // B stored transposed: B[col * n2 + row]
  B[(size_t)n * n2 + m] = make_double2(zeta * T.x, zeta * T.y);
  B[(size_t)(npsi + n) * n2 + m] = K;
  B[(size_t)n * n2 + npsi + m] = make_double2(-K.x, -K.y);
  B[(size_t)(npsi + n) * n2 + npsi + m] = make_double2(T.x / zeta, T.y / zeta);
}

// Reciprocity of the exterior blocks: T and K are symmetric bilinear forms
// (the Green's function and the triple product under the swap of source and
// test), so Z^{nu mu} = [T_nm^T ...] follows from Z^{mu nu} = [z T, K; -K, T/z]
// as Z^{nu mu}(r, c) = s_r s_c Z^{mu nu}(c, r), s = +1 on the electric rows
// and -1 on the magnetic ones.  Grid: (element chunks of 256, pairs); both
// blocks stored transposed (B[col * n2 + row]).
__global__ void k_near_mirror(int nd, int npsi, const int* __restrict__ dst, const int* __restrict__ src,
                              double2* __restrict__ Bt) {
  const int b = blockIdx.y;
  const int n2 = 2 * npsi;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nd || t >= n2 * n2) return;
  const int i = t / n2, j = t % n2;             // A(row j, col i) is A[i * n2 + j]
  const double2 a = Bt[(size_t)src[b] * n2 * n2 + (size_t)i * n2 + j];
  const double sg = ((i < npsi) == (j < npsi)) ? 1.0 : -1.0;
  Bt[(size_t)dst[b] * n2 * n2 + (size_t)j * n2 + i] = make_double2(sg * a.x, sg * a.y);
}

// Closed-form self block of a sphere (Eq. 16 with delta = 1): per (l, m) the
// transverse/longitudinal pair couples through K; T is diagonal.
static void sphere_self_block(const Shape& sh, double ko, double zo, double ki, double zi,
                              std::vector<cd>& Z) {
  int n = sh.n_psi(), n2 = 2 * n;
  Z.assign((size_t)n2 * n2, cd(0, 0));
  std::vector<int> lp, mp, kp, ll, ml, kl;
  hm::mode_list(sh.n_perp, lp, mp, kp);
  hm::mode_list(sh.n_par, ll, ml, kl);
  auto ops = [&](double kw, std::vector<cd>& T, std::vector<cd>& K) {
    T.assign((size_t)n * n, cd(0, 0));
    K.assign((size_t)n * n, cd(0, 0));
    double x = kw * sh.a;
    for (int i = 0; i < n; ++i) {
      bool perp = i < sh.n_perp;
      int l = perp ? lp[i] : ll[i - sh.n_perp];
      int m = perp ? mp[i] : ml[i - sh.n_perp];
      int kd = perp ? kp[i] : kl[i - sh.n_perp];
      double ps, dps;
      cd xi, dxi;
      hm::riccati(l, x, &ps, &dps, &xi, &dxi);
      T[(size_t)i * n + i] = perp ? -ps * xi : -dps * dxi;
      cd kk = cd(0.0, -0.5) * (ps * dxi + dps * xi);
      for (int j = 0; j < n; ++j) {
        bool perp2 = j < sh.n_perp;
        if (perp2 == perp) continue;
        int l2 = perp2 ? lp[j] : ll[j - sh.n_perp];
        int m2 = perp2 ? mp[j] : ml[j - sh.n_perp];
        int k2 = perp2 ? kp[j] : kl[j - sh.n_perp];
        if (l2 == l && m2 == m && k2 == kd) K[(size_t)i * n + j] = kk;
      }
    }
  };
  std::vector<cd> To, Ko, Ti, Ki;
  ops(ko, To, Ko);
  ops(ki, Ti, Ki);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      size_t ij = (size_t)i * n + j;
      Z[(size_t)i * n2 + j] = zo * To[ij] + zi * Ti[ij];
      Z[(size_t)i * n2 + n + j] = Ko[ij] + Ki[ij];
      Z[(size_t)(n + i) * n2 + j] = -(Ko[ij] + Ki[ij]);
      Z[(size_t)(n + i) * n2 + n + j] = To[ij] / zo + Ti[ij] / zi;
    }
}

int build_near(Ctx* c) {
  int n = c->npsi, n2 = 2 * n, S = c->S;
  int nb_total = c->nblk;   // self blocks first (S), then exterior blocks
  size_t bsz = (size_t)n2 * n2;
  std::vector<double2> selfT((size_t)S * bsz), invT((size_t)S * bsz);
  c->pinv_ok = true;
  for (int s = 0; s < S; ++s) {
    std::vector<cd> Z;
    if (c->shapes[s].rot_base >= 0) {
      Z = c->shapes[c->shapes[s].rot_base].Z;  // a rotated copy: the same self block
    } else if (c->shapes[s].mesh) {
      int rc = mesh_self_block(c, c->shapes[s], Z);
      if (rc) return rc;
    } else if (c->shapes[s].sampled) {
      Z = c->shapes[s].Z;
    } else {
      sphere_self_block(c->shapes[s], c->k, c->zeta, c->k_in, c->zeta_in, Z);
    }
    c->shapes[s].Z = Z;                        // the block in use (smr_self_block)
    std::vector<cd> Zi = Z;
    if (!hm::invert(n2, Zi)) {
      // a singular self block (possible only for shapes given as data)
      // leaves the block-diagonal preconditioner undefined; the product and
      // the unpreconditioned solve still run
      c->pinv_ok = false;
      std::fill(Zi.begin(), Zi.end(), cd(0.0, 0.0));
    }
    for (int i = 0; i < n2; ++i)
      for (int j = 0; j < n2; ++j) {
        selfT[s * bsz + (size_t)j * n2 + i] = make_double2(Z[(size_t)i * n2 + j].real(), Z[(size_t)i * n2 + j].imag());
        invT[s * bsz + (size_t)j * n2 + i] = make_double2(Zi[(size_t)i * n2 + j].real(), Zi[(size_t)i * n2 + j].imag());
      }
  }
  if (c->d_B64) cudaFree(c->d_B64);
  c->d_B64 = nullptr;
  SMR_CUDA(c, cudaMalloc((void**)&c->d_B64, (size_t)nb_total * bsz * sizeof(double2)));
  SMR_CUDA(c, cudaMemcpy(c->d_B64, selfT.data(), (size_t)S * bsz * sizeof(double2), cudaMemcpyHostToDevice));
  int rc = upload(c, &c->d_Pinv64, invT);
  if (rc) return rc;
  // exterior blocks: a block whose swapped pair (shapes exchanged, offset
  // negated) is also stored is computed once and mirrored into the other
  int nex = nb_total - S;
  if (nex > 0) {
    auto bits = [](double v) {
      if (v == 0.0) v = 0.0;                   // -0 and +0 are one key
      unsigned long long u;
      std::memcpy(&u, &v, sizeof u);
      return u;
    };
    typedef std::tuple<int, int, unsigned long long, unsigned long long, unsigned long long> Key;
    std::map<Key, int> index;
    auto off = [&](int b, int d) { return c->blk_off[3 * (size_t)(S + b) + d]; };
    for (int b = 0; b < nex; ++b)
      index[Key(c->blk_sm[S + b], c->blk_sn[S + b], bits(off(b, 0)), bits(off(b, 1)), bits(off(b, 2)))] = b;
    std::vector<int> from(nex, -1), prim, mdst, msrc;
    std::vector<char> done(nex, 0);
    for (int b = 0; b < nex; ++b) {
      if (done[b]) continue;
      done[b] = 1;
      prim.push_back(b);
      auto it = index.find(Key(c->blk_sn[S + b], c->blk_sm[S + b], bits(-off(b, 0)), bits(-off(b, 1)),
                               bits(-off(b, 2))));
      if (it != index.end() && !done[it->second]) {
        done[it->second] = 1;
        mdst.push_back(S + it->second);
        msrc.push_back(S + b);
      }
    }
    const int np = (int)prim.size();
    std::vector<int> bsm(np), bsn(np), bid(np);
    std::vector<double> bdc(3 * (size_t)np);
    for (int i = 0; i < np; ++i) {
      const int b = prim[i];
      bsm[i] = c->blk_sm[S + b];
      bsn[i] = c->blk_sn[S + b];
      bid[i] = S + b;
      for (int d = 0; d < 3; ++d) bdc[3 * (size_t)i + d] = off(b, d);
    }
    int *d_bsm = nullptr, *d_bsn = nullptr, *d_bid = nullptr, *d_md = nullptr, *d_ms = nullptr;
    double* d_bdc = nullptr;
    if ((rc = upload(c, &d_bsm, bsm)) || (rc = upload(c, &d_bsn, bsn)) || (rc = upload(c, &d_bdc, bdc)) ||
        (rc = upload(c, &d_bid, bid)) || (rc = upload(c, &d_md, mdst)) || (rc = upload(c, &d_ms, msrc)))
      return rc;
    int chunk = 64;
    double2* d_F = nullptr;
    SMR_CUDA(c, cudaMalloc((void**)&d_F, (size_t)chunk * c->Q * n * 7 * sizeof(double2)));
    for (int b0 = 0; b0 < np; b0 += chunk) {
      int nbc = std::min(chunk, np - b0);
      int qt = std::max(1, 256 / n);
      dim3 g1((c->Q + qt - 1) / qt, nbc), t1(n, qt);
      k_near_f<<<g1, t1>>>(nbc, n, c->Q, d_bsm + b0, d_bsn + b0, d_bdc + 3 * b0, c->d_modes, c->d_rq,
                           c->k, d_F);
      SMR_LAUNCH(c);
      dim3 g2((n * n + 127) / 128, nbc);
      k_near_z<<<g2, 128>>>(nbc, n, c->Q, d_bsm + b0, c->d_modes, c->d_rq, d_F, c->k, c->zeta,
                            c->d_B64, d_bid + b0);
      SMR_LAUNCH(c);
    }
    const int nm = (int)mdst.size();
    for (int m0 = 0; m0 < nm; m0 += 65535) {
      const int nd = std::min(65535, nm - m0);
      dim3 g3((unsigned)((4 * n * n + 255) / 256), (unsigned)nd);
      k_near_mirror<<<g3, 256>>>(nd, n, d_md + m0, d_ms + m0, c->d_B64);
      SMR_LAUNCH(c);
    }
    SMR_CUDA(c, cudaDeviceSynchronize());
    cudaFree(d_F);
    cudaFree(d_bsm);
    cudaFree(d_bsn);
    cudaFree(d_bdc);
    cudaFree(d_bid);
    cudaFree(d_md);
    cudaFree(d_ms);
  }
  rc = copy32(c, c->d_B64, &c->d_B32, (long long)nb_total * bsz);
  if (rc) return rc;
  return copy32(c, c->d_Pinv64, &c->d_Pinv32, (long long)S * bsz);
}

// ------------------------------------------------------------------ right-hand sides
// shape sums: Sv[s][n][c][r] = sum_q w psi_n(q) . pol_c(r) exp(-j k khat_r . r_q)
__global__ void k_rhs_shape(int S, int npsi, int Q, int R, const double* __restrict__ modes,
                            const double* __restrict__ rq, const double* __restrict__ khat,
                            const double2* __restrict__ pol, double kw, double zeta,
                            double2* __restrict__ Sv) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)S * npsi * R) return;
  int r = (int)(t % R), n = (int)((t / R) % npsi), s = (int)(t / ((long long)R * npsi));
  const double* kh = khat + 3 * r;
  const double2* e = pol + 3 * r;
  // h = khat x e / zeta
  double2 h[3];
  h[0] = make_double2((kh[1] * e[2].x - kh[2] * e[1].x) / zeta, (kh[1] * e[2].y - kh[2] * e[1].y) / zeta);
  h[1] = make_double2((kh[2] * e[0].x - kh[0] * e[2].x) / zeta, (kh[2] * e[0].y - kh[0] * e[2].y) / zeta);
  h[2] = make_double2((kh[0] * e[1].x - kh[1] * e[0].x) / zeta, (kh[0] * e[1].y - kh[1] * e[0].y) / zeta);
  const double* M = modes + ((size_t)s * npsi + n) * Q * 4;
  const double* Rr = rq + (size_t)s * Q * 4;
  double2 ae = make_double2(0, 0), ah = make_double2(0, 0);
  for (int q = 0; q < Q; ++q) {
    const double* p = Rr + 4 * q;
    const double* m = M + 4 * q;
    double sn, cs;
    sincos(-kw * (kh[0] * p[0] + kh[1] * p[1] + kh[2] * p[2]), &sn, &cs);
    double2 de = make_double2(m[0] * e[0].x + m[1] * e[1].x + m[2] * e[2].x,
                              m[0] * e[0].y + m[1] * e[1].y + m[2] * e[2].y);
    double2 dh = make_double2(m[0] * h[0].x + m[1] * h[1].x + m[2] * h[2].x,
                              m[0] * h[0].y + m[1] * h[1].y + m[2] * h[2].y);
    double w = p[3];
    ae.x += w * (de.x * cs - de.y * sn); ae.y += w * (de.x * sn + de.y * cs);
    ah.x += w * (dh.x * cs - dh.y * sn); ah.y += w * (dh.x * sn + dh.y * cs);
  }
  Sv[(((size_t)s * npsi + n) * 2 + 0) * R + r] = ae;
  Sv[(((size_t)s * npsi + n) * 2 + 1) * R + r] = ah;
}

__global__ void k_rhs_scatter(int p, int npsi, int R, const int* __restrict__ sid,
                              const double* __restrict__ cen, const double* __restrict__ khat,
                              const double2* __restrict__ Sv, double kw, double2* __restrict__ b) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p * 2 * npsi * R) return;
  int r = (int)(t % R);
  long long rest = t / R;
  int n = (int)(rest % npsi), cc = (int)((rest / npsi) % 2), mu = (int)(rest / (2 * npsi));
  const double* kh = khat + 3 * r;
  const double* x = cen + 3 * mu;
  double sn, cs;
  sincos(-kw * (kh[0] * x[0] + kh[1] * x[1] + kh[2] * x[2]), &sn, &cs);
  double2 v = Sv[(((size_t)sid[mu] * npsi + n) * 2 + cc) * R + r];
  b[t] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
}

int launch_rhs(Ctx* c, int R, const double* d_khat, const double2* d_pol, double2* b,
               cudaStream_t st) {
  double2* Sv = nullptr;
  SMR_CUDA(c, cudaMallocAsync((void**)&Sv, (size_t)c->S * c->npsi * 2 * R * sizeof(double2), st));
  long long t1 = (long long)c->S * c->npsi * R;
  k_rhs_shape<<<(unsigned)((t1 + 127) / 128), 128, 0, st>>>(c->S, c->npsi, c->Q, R, c->d_modes, c->d_rq,
                                                           d_khat, d_pol, c->k, c->zeta, Sv);
  SMR_LAUNCH(c);
  long long t2 = (long long)c->p * 2 * c->npsi * R;
  k_rhs_scatter<<<(unsigned)((t2 + 255) / 256), 256, 0, st>>>(c->p, c->npsi, R, c->d_sid, c->d_centres,
                                                             d_khat, Sv, c->k, b);
  SMR_LAUNCH(c);
  SMR_CUDA(c, cudaFreeAsync(Sv, st));
  return SMR_OK;
}

// per-array incidence: b[mu][c][n] = exp(-j k khat_a . r_mu) Sv[s_mu][n][c][a], a = arr[mu]
__global__ void k_rhs_scatter_arrays(int p, int npsi, int na, const int* __restrict__ sid,
                                     const int* __restrict__ arr, const double* __restrict__ cen,
                                     const double* __restrict__ khat, const double2* __restrict__ Sv,
                                     double kw, double2* __restrict__ b) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p * 2 * npsi) return;
  int n = (int)(t % npsi), cc = (int)((t / npsi) % 2), mu = (int)(t / (2 * npsi));
  int a = arr[mu];
  const double* kh = khat + 3 * a;
  const double* x = cen + 3 * mu;
  double sn, cs;
  sincos(-kw * (kh[0] * x[0] + kh[1] * x[1] + kh[2] * x[2]), &sn, &cs);
  double2 v = Sv[(((size_t)sid[mu] * npsi + n) * 2 + cc) * na + a];
  b[t] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
}

int launch_rhs_arrays(Ctx* c, const double* d_khat, const double2* d_pol, double2* b, cudaStream_t st) {
  int na = c->n_arrays;
  double2* Sv = nullptr;
  SMR_CUDA(c, cudaMallocAsync((void**)&Sv, (size_t)c->S * c->npsi * 2 * na * sizeof(double2), st));
  long long t1 = (long long)c->S * c->npsi * na;
  k_rhs_shape<<<(unsigned)((t1 + 127) / 128), 128, 0, st>>>(c->S, c->npsi, c->Q, na, c->d_modes, c->d_rq,
                                                           d_khat, d_pol, c->k, c->zeta, Sv);
  SMR_LAUNCH(c);
  long long t2 = (long long)c->p * 2 * c->npsi;
  k_rhs_scatter_arrays<<<(unsigned)((t2 + 255) / 256), 256, 0, st>>>(c->p, c->npsi, na, c->d_sid, c->d_arr,
                                                                    c->d_centres, d_khat, Sv, c->k, b);
  SMR_LAUNCH(c);
  SMR_CUDA(c, cudaFreeAsync(Sv, st));
  return SMR_OK;
}

// Same two kernels with caller-provided scratch Sv [S][n_psi][2][R] (no allocation).
int launch_rhs_scratch(Ctx* c, int R, const double* d_khat, const double2* d_pol, double2* Sv,
                       double2* b, cudaStream_t st) {
  long long t1 = (long long)c->S * c->npsi * R;
  k_rhs_shape<<<(unsigned)((t1 + 127) / 128), 128, 0, st>>>(c->S, c->npsi, c->Q, R, c->d_modes, c->d_rq,
                                                           d_khat, d_pol, c->k, c->zeta, Sv);
  SMR_LAUNCH(c);
  long long t2 = (long long)c->p * 2 * c->npsi * R;
  k_rhs_scatter<<<(unsigned)((t2 + 255) / 256), 256, 0, st>>>(c->p, c->npsi, R, c->d_sid, c->d_centres,
                                                             d_khat, Sv, c->k, b);
  SMR_LAUNCH(c);
  return SMR_OK;
}

// ------------------------------------------------------------------ far field
// Rv[s][n][d][3] = sum_q w psi_n(q) exp(+j k rhat_d . r_q)   (radiation vectors)
__global__ void k_radvec(int S, int npsi, int Q, int nd, const double* __restrict__ modes,
                         const double* __restrict__ rq, const double* __restrict__ dirs, double kw,
                         double2* __restrict__ Rv) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)S * npsi * nd) return;
  int d = (int)(t % nd), n = (int)((t / nd) % npsi), s = (int)(t / ((long long)nd * npsi));
  const double* u = dirs + 3 * d;
  const double* M = modes + ((size_t)s * npsi + n) * Q * 4;
  const double* Rr = rq + (size_t)s * Q * 4;
  double2 a[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int q = 0; q < Q; ++q) {
    const double* p = Rr + 4 * q;
    double sn, cs;
    sincos(kw * (u[0] * p[0] + u[1] * p[1] + u[2] * p[2]), &sn, &cs);
    for (int i = 0; i < 3; ++i) {
      double v = p[3] * M[4 * q + i];
      a[i].x += v * cs;
      a[i].y += v * sn;
    }
  }
  for (int i = 0; i < 3; ++i) Rv[t * 3 + i] = a[i];
}

// F[d][3][r]: CTA per (d, r); threads stride over particles; block reduction.
__global__ void k_farfield(int p, int npsi, int nd, int R, const int* __restrict__ sid,
                           const double* __restrict__ cen, const double* __restrict__ dirs,
                           const double2* __restrict__ Rv, const double2* __restrict__ x,
                           double kw, double zeta, double2* __restrict__ F) {
  int d = blockIdx.x / R, r = blockIdx.x % R;
  const double* u = dirs + 3 * d;
  double2 J[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  double2 M[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int mu = threadIdx.x; mu < p; mu += blockDim.x) {
    const double* cc = cen + 3 * mu;
    double sn, cs;
    sincos(kw * (u[0] * cc[0] + u[1] * cc[1] + u[2] * cc[2]), &sn, &cs);
    int s = sid[mu];
    double2 je[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    double2 jm[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int n = 0; n < npsi; ++n) {
      double2 ae = x[((size_t)mu * 2 * npsi + n) * R + r];
      double2 am = x[((size_t)mu * 2 * npsi + npsi + n) * R + r];
      const double2* rv = Rv + (((size_t)s * npsi + n) * nd + d) * 3;
      for (int i = 0; i < 3; ++i) {
        je[i].x += ae.x * rv[i].x - ae.y * rv[i].y; je[i].y += ae.x * rv[i].y + ae.y * rv[i].x;
        jm[i].x += am.x * rv[i].x - am.y * rv[i].y; jm[i].y += am.x * rv[i].y + am.y * rv[i].x;
      }
    }
    for (int i = 0; i < 3; ++i) {
      J[i].x += je[i].x * cs - je[i].y * sn; J[i].y += je[i].x * sn + je[i].y * cs;
      M[i].x += jm[i].x * cs - jm[i].y * sn; M[i].y += jm[i].x * sn + jm[i].y * cs;
    }
  }
  __shared__ double red[12][256];
  for (int i = 0; i < 3; ++i) {
    red[2 * i][threadIdx.x] = J[i].x; red[2 * i + 1][threadIdx.x] = J[i].y;
    red[6 + 2 * i][threadIdx.x] = M[i].x; red[7 + 2 * i][threadIdx.x] = M[i].y;
  }
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < 12; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double2 Jt[3], Mt[3];
  for (int i = 0; i < 3; ++i) {
    Jt[i] = make_double2(red[2 * i][0], red[2 * i + 1][0]);
    Mt[i] = make_double2(red[6 + 2 * i][0], red[7 + 2 * i][0]);
  }
  double2 rj = make_double2(u[0] * Jt[0].x + u[1] * Jt[1].x + u[2] * Jt[2].x,
                            u[0] * Jt[0].y + u[1] * Jt[1].y + u[2] * Jt[2].y);
  double2 rxm[3];
  rxm[0] = make_double2(u[1] * Mt[2].x - u[2] * Mt[1].x, u[1] * Mt[2].y - u[2] * Mt[1].y);
  rxm[1] = make_double2(u[2] * Mt[0].x - u[0] * Mt[2].x, u[2] * Mt[0].y - u[0] * Mt[2].y);
  rxm[2] = make_double2(u[0] * Mt[1].x - u[1] * Mt[0].x, u[0] * Mt[1].y - u[1] * Mt[0].y);
  double pre = kw / (4.0 * PI);  // F = j pre [ zeta (J - u (u.J)) - u x M ]
  for (int i = 0; i < 3; ++i) {
    double vx = zeta * (Jt[i].x - u[i] * rj.x) - rxm[i].x;
    double vy = zeta * (Jt[i].y - u[i] * rj.y) - rxm[i].y;
    F[((size_t)d * 3 + i) * R + r] = make_double2(-pre * vy, pre * vx);
  }
}

int launch_far_field(Ctx* c, int R, const double2* x, int nd, const double* d_dirs, double2* F,
                     cudaStream_t st) {
  double2* Rv = nullptr;
  SMR_CUDA(c, cudaMallocAsync((void**)&Rv, (size_t)c->S * c->npsi * nd * 3 * sizeof(double2), st));
  long long t1 = (long long)c->S * c->npsi * nd;
  k_radvec<<<(unsigned)((t1 + 127) / 128), 128, 0, st>>>(c->S, c->npsi, c->Q, nd, c->d_modes, c->d_rq,
                                                        d_dirs, c->k, Rv);
  SMR_LAUNCH(c);
  k_farfield<<<(unsigned)(nd * R), 256, 0, st>>>(c->p, c->npsi, nd, R, c->d_sid, c->d_centres, d_dirs,
                                                 Rv, x, c->k, c->zeta, F);
  SMR_LAUNCH(c);
  SMR_CUDA(c, cudaFreeAsync(Rv, st));
  return SMR_OK;
}

// Cross sections from far-field amplitudes F[nd][3][R].  CTA per column r:
// the first n_sca directions carry quadrature weights W (scattered power
// over the sphere, Sec. V); direction n_sca + r is column r's own incident
// direction, where the optical theorem gives the extinction.  cs[2r] = C_sca,
// cs[2r + 1] = C_ext.
__global__ void k_cross_sections(int n_sca, int R, const double2* __restrict__ F,
                                 const double* __restrict__ W, const double2* __restrict__ pol,
                                 double kw, double* __restrict__ cs) {
  __shared__ double red[256];
  int r = blockIdx.x;
  double acc = 0;
  for (int d = threadIdx.x; d < n_sca; d += blockDim.x) {
    double e = 0;
    for (int i = 0; i < 3; ++i) {
      double2 f = F[((size_t)d * 3 + i) * R + r];
      e += f.x * f.x + f.y * f.y;
    }
    acc += W[d] * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // Im(conj(e) . F) / |e|^2 at the forward direction.
    double im = 0, nn = 0;
    for (int i = 0; i < 3; ++i) {
      double2 e = pol[(size_t)r * 3 + i];
      double2 f = F[((size_t)(n_sca + r) * 3 + i) * R + r];
      im += e.x * f.y - e.y * f.x;
      nn += e.x * e.x + e.y * e.y;
    }
    cs[2 * r] = red[0];
    cs[2 * r + 1] = -(4.0 * M_PI / kw) * im / nn;
  }
}

int launch_cross_sections(Ctx* c, int R, const double2* x, int n_sca, const double* d_dirs,
                          const double* d_w, const double2* d_pol, double* d_cs, cudaStream_t st) {
  int nd = n_sca + R;
  double2* F = nullptr;
  SMR_CUDA(c, cudaMallocAsync((void**)&F, (size_t)nd * 3 * R * sizeof(double2), st));
  int rc = launch_far_field(c, R, x, nd, d_dirs, F, st);
  if (rc == SMR_OK) {
    k_cross_sections<<<R, 256, 0, st>>>(n_sca, R, F, d_w, d_pol, c->k, d_cs);
    SMR_LAUNCH(c);
  }
  SMR_CUDA(c, cudaFreeAsync(F, st));
  return rc;
}

// ------------------------------------------------------------------ near field
// CTA per particle mu (and right-hand side r): currents at the quadrature
// points staged in shared memory; threads stride over field points and add
// their particle's contribution with atomics.
// Field points in groups of blockDim (one point per thread, blockIdx.z),
// one right-hand side per blockIdx.y; the blocks of a group stride over the
// units (particle, chunk of at most QC surface points): each unit's currents
// are staged in shared memory and every thread adds their field at its point
// in registers.  One atomic add per block and field component at the end.
__global__ void k_nearfield(int p, int npsi, int Q, int QC, int npt, int R, const int* __restrict__ sid,
                            const double* __restrict__ cen, const double* __restrict__ modes,
                            const double* __restrict__ rq, const double2* __restrict__ x,
                            const double* __restrict__ pts, double kw, double zeta,
                            double* __restrict__ EH) {
  extern __shared__ double sm[];   // [QC][8 complex] J xyz, divJ, M xyz, divM  + [QC][4] point
  const int nch = (Q + QC - 1) / QC;
  const int r = blockIdx.y;
  const int ip = blockIdx.z * blockDim.x + threadIdx.x;
  const bool act = ip < npt;
  double2* cur = reinterpret_cast<double2*>(sm);
  double* pq = sm + (size_t)QC * 16;
  double P[3] = {0, 0, 0};
  if (act)
    for (int d = 0; d < 3; ++d) P[d] = pts[3 * ip + d];
  double2 E[3], H[3];
  for (int i = 0; i < 3; ++i) { E[i] = make_double2(0, 0); H[i] = make_double2(0, 0); }
  for (long long u = blockIdx.x; u < (long long)p * nch; u += gridDim.x) {
    const int mu = (int)(u / nch), ch = (int)(u % nch);
    const int s = sid[mu];
    const int q0 = ch * QC, nq = min(QC, Q - q0);
    const double* Ms = modes + (size_t)s * npsi * Q * 4 + (size_t)q0 * 4;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      double2 a[8];
      for (int i = 0; i < 8; ++i) a[i] = make_double2(0, 0);
      for (int n = 0; n < npsi; ++n) {
        double2 ae = x[((size_t)mu * 2 * npsi + n) * R + r];
        double2 am = x[((size_t)mu * 2 * npsi + npsi + n) * R + r];
        const double* m = Ms + ((size_t)n * Q + q) * 4;
        for (int i = 0; i < 4; ++i) {
          a[i].x += ae.x * m[i]; a[i].y += ae.y * m[i];
          a[4 + i].x += am.x * m[i]; a[4 + i].y += am.y * m[i];
        }
      }
      for (int i = 0; i < 8; ++i) cur[(size_t)q * 8 + i] = a[i];
      const double* rr = rq + ((size_t)s * Q + q0 + q) * 4;
      pq[4 * q] = rr[0] + cen[3 * mu];
      pq[4 * q + 1] = rr[1] + cen[3 * mu + 1];
      pq[4 * q + 2] = rr[2] + cen[3 * mu + 2];
      pq[4 * q + 3] = rr[3];
    }
    __syncthreads();
    if (act) {
      for (int q = 0; q < nq; ++q) {
        double d[3] = {P[0] - pq[4 * q], P[1] - pq[4 * q + 1], P[2] - pq[4 * q + 2]};
        double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double Rr = sqrt(R2), iR = 1.0 / Rr;
        double sn, cs;
        sincos(-kw * Rr, &sn, &cs);
        double w = pq[4 * q + 3];
        double g = w * iR / (4.0 * PI);
        double2 G = make_double2(g * cs, g * sn);
        // grad_r g = -(d) (1 + jkR) e / (4 pi R^3)   (times w)
        double g3 = g * iR * iR;
        double2 D = make_double2(-g3 * (cs - kw * Rr * sn), -g3 * (sn + kw * Rr * cs));
        const double2* c8 = cur + (size_t)q * 8;
        for (int which = 0; which < 2; ++which) {
          const double2* X = c8 + 4 * which;
          // L{X} = -jk G X - (j/k) grad g (div X)
          // K{X} = grad g x X
          double2 Lv[3], Kv[3];
          double2 DX = make_double2(D.x * X[3].x - D.y * X[3].y, D.x * X[3].y + D.y * X[3].x);
          for (int i = 0; i < 3; ++i) {
            double2 GX = make_double2(G.x * X[i].x - G.y * X[i].y, G.x * X[i].y + G.y * X[i].x);
            // -jk GX - (j/k) d_i DX
            Lv[i] = make_double2(kw * GX.y + d[i] * DX.y / kw, -kw * GX.x - d[i] * DX.x / kw);
          }
          // (d x X) * D
          double2 cxX[3];
          cxX[0] = make_double2(d[1] * X[2].x - d[2] * X[1].x, d[1] * X[2].y - d[2] * X[1].y);
          cxX[1] = make_double2(d[2] * X[0].x - d[0] * X[2].x, d[2] * X[0].y - d[0] * X[2].y);
          cxX[2] = make_double2(d[0] * X[1].x - d[1] * X[0].x, d[0] * X[1].y - d[1] * X[0].y);
          for (int i = 0; i < 3; ++i)
            Kv[i] = make_double2(D.x * cxX[i].x - D.y * cxX[i].y, D.x * cxX[i].y + D.y * cxX[i].x);
          if (which == 0) {  // J: E += -zeta L{J}, H += -K{J}
            for (int i = 0; i < 3; ++i) {
              E[i].x -= zeta * Lv[i].x; E[i].y -= zeta * Lv[i].y;
              H[i].x -= Kv[i].x; H[i].y -= Kv[i].y;
            }
          } else {           // M: E += K{M}, H += -L{M}/zeta
            for (int i = 0; i < 3; ++i) {
              E[i].x += Kv[i].x; E[i].y += Kv[i].y;
              H[i].x -= Lv[i].x / zeta; H[i].y -= Lv[i].y / zeta;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if (act) {
    double* o = EH + (((size_t)ip * 6) * R + r) * 2;
    for (int i = 0; i < 3; ++i) {
      atomicAdd(o + ((size_t)i * R) * 2, E[i].x);
      atomicAdd(o + ((size_t)i * R) * 2 + 1, E[i].y);
      atomicAdd(o + ((size_t)(3 + i) * R) * 2, H[i].x);
      atomicAdd(o + ((size_t)(3 + i) * R) * 2 + 1, H[i].y);
    }
  }
}

int launch_near_field(Ctx* c, int R, const double2* x, int npt, const double* d_pts, double2* EH,
                      cudaStream_t st) {
  SMR_CUDA(c, cudaMemsetAsync(EH, 0, (size_t)npt * 6 * R * sizeof(double2), st));
  const int QC = std::min(c->Q, 1024);
  const int nch = (c->Q + QC - 1) / QC;
  size_t sm = (size_t)QC * (16 + 4) * sizeof(double);
  SMR_CUDA(c, cudaFuncSetAttribute(k_nearfield, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  const long long units = (long long)c->p * nch;
  dim3 grid((unsigned)std::min<long long>(units, 1216), (unsigned)R, (unsigned)((npt + 255) / 256));
  k_nearfield<<<grid, 256, sm, st>>>(c->p, c->npsi, c->Q, QC, npt, R, c->d_sid, c->d_centres, c->d_modes,
                                     c->d_rq, x, d_pts, c->k, c->zeta, (double*)EH);
  SMR_LAUNCH(c);
  return SMR_OK;
}

}  // namespace smr
