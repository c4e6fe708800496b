// Hot path of the MLFMA-SMR product (Sec. IV): near block-sparse product,
// aggregation, interpolation, translation, anterpolation and receive.
// Every kernel is templated on the arithmetic type (double / float); the
// unknown vectors stay complex FP64 and are converted on load / store.
//
// Layouts (complex, interleaved):
//   x, y              [p][2][n_psi][R]
//   patterns P        [S][n_psi][2][K0]       (theta, phi components, Eq. 26)
//   spectra out/in    [n_box][K_s][4][R]      fields A_e.th, A_e.ph, A_m.th, A_m.ph
//   translation T     [n_offset][K_s]         (Eq. 23)
//   near blocks       [n_blk][2 n_psi (col j)][2 n_psi (row i)]  (transposed)
#include <algorithm>

#include "smr_internal.h"

namespace smr {

template <typename T> struct CV;
template <> struct CV<double> { typedef double2 V; };
template <> struct CV<float> { typedef float2 V; };

__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
template <typename V> __device__ __forceinline__ V czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 cvt2(double2 v, double2) { return v; }
__device__ __forceinline__ float2 cvt2(double2 v, float2) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to64(double2 v) { return v; }
__device__ __forceinline__ double2 to64(float2 v) { return make_double2(v.x, v.y); }

// acc += a * b
template <typename V> __device__ __forceinline__ void cfma(V& acc, V a, V b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename V> __device__ __forceinline__ void cfmac(V& acc, V a, V b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += w * b  (w real)
template <typename V, typename T> __device__ __forceinline__ void rfma(V& acc, T w, V b) {
  acc.x = fma(w, b.x, acc.x);
  acc.y = fma(w, b.y, acc.y);
}
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// ------------------------------------------------------------------ aggregation
// out0[mu][k][f][r] = shift * sum_n conj(P[s][n][comp f][k]) x[mu][cur f][n][r]
template <typename T>
__global__ void k_aggregate(int p, int K0, int npsi, int R, int kc, int nchunk,
                            const double2* __restrict__ x, const typename CV<T>::V* __restrict__ P,
                            const int* __restrict__ sid, const double* __restrict__ dshift,
                            int any_dshift, const double* __restrict__ khat, double k,
                            typename CV<T>::V* __restrict__ out) {
  typedef typename CV<T>::V V;
  int mu = blockIdx.x / nchunk, chunk = blockIdx.x % nchunk;
  int kl = threadIdx.x / R, r = threadIdx.x % R;
  if (kl >= kc) return;
  int kk = chunk * kc + kl;
  if (kk >= K0) return;
  const V* Ps = P + (size_t)sid[mu] * npsi * 2 * K0 + kk;
  const double2* xe = x + (size_t)mu * 2 * npsi * R + r;
  const double2* xm = xe + (size_t)npsi * R;
  V a0 = czero<V>(), a1 = czero<V>(), a2 = czero<V>(), a3 = czero<V>();
  for (int n = 0; n < npsi; ++n) {
    V pt = Ps[(size_t)(2 * n) * K0], pp = Ps[(size_t)(2 * n + 1) * K0];
    V e = cvt2(xe[(size_t)n * R], V()), m = cvt2(xm[(size_t)n * R], V());
    cfmac(a0, pt, e);
    cfmac(a1, pp, e);
    cfmac(a2, pt, m);
    cfmac(a3, pp, m);
  }
  if (any_dshift) {
    const double* d = dshift + 3 * mu;
    const double* kh = khat + 3 * kk;
    double ph = k * (kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2]);
    double sn, cs;
    sincos(ph, &sn, &cs);
    V sh = mkc((T)cs, (T)sn);
    a0 = cmul(a0, sh); a1 = cmul(a1, sh); a2 = cmul(a2, sh); a3 = cmul(a3, sh);
  }
  V* o = out + ((size_t)mu * K0 + kk) * 4 * R + r;
  o[0] = a0; o[R] = a1; o[2 * R] = a2; o[3 * R] = a3;
}

// ------------------------------------------------------------------ interpolation
// outP[B][kp] = sum_children shift[q][kp] * sum_{4x4 taps} w sgn outC[c][tap]
template <typename T>
__global__ void k_interp(int nboxP, int Kp, int nphP, int nphC, int Kc, int R, int kc,
                         const int* __restrict__ ch_ptr, const int* __restrict__ ch_idx,
                         const int* __restrict__ ch_quad, const int* __restrict__ th_src,
                         const int* __restrict__ th_refl, const T* __restrict__ th_w,
                         const int* __restrict__ ph_src, const T* __restrict__ ph_w,
                         const typename CV<T>::V* __restrict__ shift,
                         const typename CV<T>::V* __restrict__ outC,
                         typename CV<T>::V* __restrict__ outP) {
  typedef typename CV<T>::V V;
  int B = blockIdx.x % nboxP, chunk = blockIdx.x / nboxP;
  int kl = threadIdx.x / R, r = threadIdx.x % R;
  if (kl >= kc) return;
  int kp = chunk * kc + kl;
  if (kp >= Kp) return;
  int tp = kp / nphP, jp = kp - tp * nphP;
  int rowoff[4], colA[4], colB[4];
  T wt[4], wp[4];
  for (int a = 0; a < 4; ++a) {
    int refl = th_refl[tp * 4 + a];
    rowoff[a] = th_src[tp * 4 + a] * nphC;
    wt[a] = refl ? -th_w[tp * 4 + a] : th_w[tp * 4 + a];
    colA[a] = refl;  // reuse as flag
  }
  int half = nphC / 2;
  for (int b = 0; b < 4; ++b) {
    int j = ph_src[jp * 4 + b];
    wp[b] = ph_w[jp * 4 + b];
    colB[b] = j;
  }
  V acc[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
  for (int e = ch_ptr[B]; e < ch_ptr[B + 1]; ++e) {
    const V* src = outC + (size_t)ch_idx[e] * Kc * 4 * R + r;
    V t[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
    for (int a = 0; a < 4; ++a) {
      for (int b = 0; b < 4; ++b) {
        int col = colA[a] ? (colB[b] + half) % nphC : colB[b];
        T w = wt[a] * wp[b];
        const V* s = src + (size_t)(rowoff[a] + col) * 4 * R;
        rfma(t[0], w, s[0]);
        rfma(t[1], w, s[R]);
        rfma(t[2], w, s[2 * R]);
        rfma(t[3], w, s[3 * R]);
      }
    }
    V sh = shift[(size_t)ch_quad[e] * Kp + kp];
    for (int f = 0; f < 4; ++f) cfma(acc[f], sh, t[f]);
  }
  V* o = outP + ((size_t)B * Kp + kp) * 4 * R + r;
  for (int f = 0; f < 4; ++f) o[f * R] = acc[f];
}

// ------------------------------------------------------------------ translation
// in[b][k] = sum_{(b', o) in IL(b)} T[o][k] out[b'][k]   (Eqs. 22-23)
template <typename T>
__global__ void k_translate(int nbox, int K, int R, int kc, const int* __restrict__ il_ptr,
                            const int* __restrict__ il_src, const int* __restrict__ il_off,
                            const typename CV<T>::V* __restrict__ Tt,
                            const typename CV<T>::V* __restrict__ out,
                            typename CV<T>::V* __restrict__ in) {
  typedef typename CV<T>::V V;
  int b = blockIdx.x % nbox, chunk = blockIdx.x / nbox;
  int kl = threadIdx.x / R, r = threadIdx.x % R;
  if (kl >= kc) return;
  int kk = chunk * kc + kl;
  if (kk >= K) return;
  V acc[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
  for (int e = il_ptr[b]; e < il_ptr[b + 1]; ++e) {
    V t = Tt[(size_t)il_off[e] * K + kk];
    const V* s = out + ((size_t)il_src[e] * K + kk) * 4 * R + r;
    cfma(acc[0], t, s[0]);
    cfma(acc[1], t, s[R]);
    cfma(acc[2], t, s[2 * R]);
    cfma(acc[3], t, s[3 * R]);
  }
  V* o = in + ((size_t)b * K + kk) * 4 * R + r;
  for (int f = 0; f < 4; ++f) o[f * R] = acc[f];
}

// ------------------------------------------------------------------ anterpolation
// inC[c][kc] += sum_{(kp, w) in A(kc)} w conj(shift[q][kp]) inP[parent][kp]
template <typename T>
__global__ void k_anterp(int nboxC, int Kc, int Kp, int R, int kc, const int* __restrict__ parent,
                         const int* __restrict__ quad, const int* __restrict__ ant_ptr,
                         const int* __restrict__ ant_idx, const T* __restrict__ ant_w,
                         const typename CV<T>::V* __restrict__ shift,
                         const typename CV<T>::V* __restrict__ inP,
                         typename CV<T>::V* __restrict__ inC) {
  typedef typename CV<T>::V V;
  int c = blockIdx.x % nboxC, chunk = blockIdx.x / nboxC;
  int kl = threadIdx.x / R, r = threadIdx.x % R;
  if (kl >= kc) return;
  int kk = chunk * kc + kl;
  if (kk >= Kc) return;
  const V* sh = shift + (size_t)quad[c] * Kp;
  const V* src = inP + (size_t)parent[c] * Kp * 4 * R + r;
  V acc[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
  for (int e = ant_ptr[kk]; e < ant_ptr[kk + 1]; ++e) {
    int kp = ant_idx[e];
    T w = ant_w[e];
    V s = sh[kp];
    V cw = mkc(w * s.x, -w * s.y);   // w conj(shift)
    const V* v = src + (size_t)kp * 4 * R;
    cfma(acc[0], cw, v[0]);
    cfma(acc[1], cw, v[R]);
    cfma(acc[2], cw, v[2 * R]);
    cfma(acc[3], cw, v[3 * R]);
  }
  V* o = inC + ((size_t)c * Kc + kk) * 4 * R + r;
  for (int f = 0; f < 4; ++f) {
    V cur = o[f * R];
    cur.x += acc[f].x;
    cur.y += acc[f].y;
    o[f * R] = cur;
  }
}

// ------------------------------------------------------------------ receive
// y_e[m] += -jk sum_k w conj(sh) [P_th (z B0 + B3) + P_ph (z B1 - B2)]
// y_m[m] += -jk sum_k w conj(sh) [P_th (-B1 + B2/z) + P_ph (B0 + B3/z)]   (Eqs. 24-25)
template <typename T>
__global__ void k_receive(int p, int K0, int npsi, int R, int rc, int nrc,
                          const typename CV<T>::V* __restrict__ in0,
                          const typename CV<T>::V* __restrict__ P, const int* __restrict__ sid,
                          const double* __restrict__ w0, const double* __restrict__ dshift,
                          int any_dshift, const double* __restrict__ khat, double k, double zeta,
                          double2* __restrict__ y, int accumulate) {
  typedef typename CV<T>::V V;
  extern __shared__ unsigned char smem_raw[];
  V* Bs = reinterpret_cast<V*>(smem_raw);           // [K0][4][rc]
  int mu = blockIdx.x / nrc, r0 = (blockIdx.x % nrc) * rc;
  int nr = min(rc, R - r0);
  const V* src = in0 + (size_t)mu * K0 * 4 * R;
  for (int t = threadIdx.x; t < K0 * 4 * nr; t += blockDim.x) {
    int rl = t % nr, f = (t / nr) % 4, kk = t / (4 * nr);
    V v = src[((size_t)kk * 4 + f) * R + r0 + rl];
    T wk = (T)w0[kk];
    v.x *= wk;
    v.y *= wk;
    if (any_dshift) {
      const double* d = dshift + 3 * mu;
      const double* kh = khat + 3 * kk;
      double ph = -k * (kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2]);
      double sn, cs;
      sincos(ph, &sn, &cs);
      v = cmul(v, mkc((T)cs, (T)sn));
    }
    Bs[((size_t)kk * 4 + f) * rc + rl] = v;
  }
  __syncthreads();
  int m = threadIdx.x / rc, rl = threadIdx.x % rc;
  if (m >= npsi || rl >= nr) return;
  const V* Pm = P + ((size_t)sid[mu] * npsi + m) * 2 * K0;
  T z = (T)zeta, iz = (T)(1.0 / zeta);
  V ye = czero<V>(), ym = czero<V>();
  for (int kk = 0; kk < K0; ++kk) {
    V pt = Pm[kk], pp = Pm[K0 + kk];
    const V* Bk = Bs + (size_t)kk * 4 * rc + rl;
    V B0 = Bk[0], B1 = Bk[rc], B2 = Bk[2 * rc], B3 = Bk[3 * rc];
    V e1 = mkc(z * B0.x + B3.x, z * B0.y + B3.y);
    V e2 = mkc(z * B1.x - B2.x, z * B1.y - B2.y);
    V m1 = mkc(-B1.x + iz * B2.x, -B1.y + iz * B2.y);
    V m2 = mkc(B0.x + iz * B3.x, B0.y + iz * B3.y);
    cfma(ye, pt, e1);
    cfma(ye, pp, e2);
    cfma(ym, pt, m1);
    cfma(ym, pp, m2);
  }
  // multiply by -j k
  double2 oe = make_double2(k * (double)ye.y, -k * (double)ye.x);
  double2 om = make_double2(k * (double)ym.y, -k * (double)ym.x);
  double2* ye_p = y + ((size_t)mu * 2 * npsi + m) * R + r0 + rl;
  double2* ym_p = ye_p + (size_t)npsi * R;
  if (accumulate) {
    double2 a = *ye_p, b = *ym_p;
    oe.x += a.x; oe.y += a.y; om.x += b.x; om.y += b.y;
  }
  *ye_p = oe;
  *ym_p = om;
}

// ------------------------------------------------------------------ block-sparse product
// y[mu][i][r] (+)= sum_{e in row mu} sum_j B[blk_e][i][j] x[col_e][j][r]
template <typename T>
__global__ void k_blocksparse(int nrow, int n2, int R, int rc, int nrc, const int* __restrict__ ptr,
                              const int* __restrict__ col, const int* __restrict__ blk,
                              const typename CV<T>::V* __restrict__ Bt,
                              const double2* __restrict__ x, double2* __restrict__ y,
                              int accumulate) {
  typedef typename CV<T>::V V;
  extern __shared__ unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);            // [n2][rc]
  int mu = blockIdx.x / nrc, r0 = (blockIdx.x % nrc) * rc;
  int nr = min(rc, R - r0);
  int i = threadIdx.x / rc, rl = threadIdx.x % rc;
  bool active = (i < n2) && (rl < nr);
  V acc = czero<V>();
  for (int e = ptr[mu]; e < ptr[mu + 1]; ++e) {
    const double2* xv = x + (size_t)col[e] * n2 * R + r0;
    __syncthreads();
    for (int t = threadIdx.x; t < n2 * nr; t += blockDim.x) {
      int jl = t / nr, q = t % nr;
      xs[jl * rc + q] = cvt2(xv[(size_t)jl * R + q], V());
    }
    __syncthreads();
    if (active) {
      const V* Bb = Bt + (size_t)blk[e] * n2 * n2 + i;
      for (int j = 0; j < n2; ++j) cfma(acc, Bb[(size_t)j * n2], xs[j * rc + rl]);
    }
  }
  if (!active) return;
  double2* yp = y + ((size_t)mu * n2 + i) * R + r0 + rl;
  double2 o = to64(acc);
  if (accumulate) {
    double2 a = *yp;
    o.x += a.x;
    o.y += a.y;
  }
  *yp = o;
}

// ------------------------------------------------------------------ host drivers
static inline int kchunk(int R) { return std::max(1, 256 / R); }

int ensure_spectra(Ctx* c, int R, int prec) {
  if (c->spec_R == R && c->spec_prec == prec) return SMR_OK;
  size_t es = (prec == SMR_PREC_FP64) ? sizeof(double2) : sizeof(float2);
  for (auto& L : c->lev) {
    if (L.d_out) cudaFree(L.d_out);
    if (L.d_in) cudaFree(L.d_in);
    L.d_out = L.d_in = nullptr;
    size_t bytes = (size_t)L.nbox * L.K * 4 * R * es;
    if (cudaMalloc(&L.d_out, bytes) != cudaSuccess || cudaMalloc(&L.d_in, bytes) != cudaSuccess) {
      c->err = "out of device memory for level spectra";
      c->spec_R = 0;
      c->spec_prec = -1;
      return SMR_E_OOM;
    }
    L.spec_bytes = bytes;
  }
  c->spec_R = R;
  c->spec_prec = prec;
  return SMR_OK;
}

template <typename T>
static int far_impl(Ctx* c, int R, const double2* x, double2* y, bool accumulate, cudaStream_t st) {
  typedef typename CV<T>::V V;
  const bool f64 = sizeof(T) == 8;
  int kc = kchunk(R);
  Level& L0 = c->lev[0];
  // aggregation
  const double es = sizeof(V), R_ = R;
  {
    int nchunk = (L0.K + kc - 1) / kc;
    pbeg(c, st, "aggregate", 0,
         (double)c->p * 2 * c->npsi * R_ * 16 + (double)c->S * c->npsi * 2 * L0.K * es +
             (double)c->p * L0.K * 4 * R_ * es,
         32.0 * c->npsi * c->p * L0.K * R_);
    k_aggregate<T><<<(unsigned)(c->p * nchunk), 256, 0, st>>>(
        c->p, L0.K, c->npsi, R, kc, nchunk, x, (const V*)(f64 ? (void*)c->d_P64 : (void*)c->d_P32),
        c->d_sid, c->d_dshift, c->any_dshift, L0.d_khat, c->k, (V*)L0.d_out);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  // upward
  for (int s = 0; s + 1 < c->nlev; ++s) {
    Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
    int nchunk = (Lp.K + kc - 1) / kc;
    pbeg(c, st, "interpolate", s,
         ((double)Lc.nbox * Lc.K + (double)Lp.nbox * Lp.K) * 4 * R_ * es + 4.0 * Lp.K * es,
         (double)Lc.nbox * Lp.K * 4 * R_ * 72.0);
    k_interp<T><<<(unsigned)(Lp.nbox * nchunk), 256, 0, st>>>(
        Lp.nbox, Lp.K, Lp.nph, Lc.nph, Lc.K, R, kc, Lp.d_ch_ptr, Lp.d_ch_idx, Lp.d_ch_quad,
        Lc.d_th_src, Lc.d_th_refl, (const T*)(f64 ? (void*)Lc.d_th_w64 : (void*)Lc.d_th_w32),
        Lc.d_ph_src, (const T*)(f64 ? (void*)Lc.d_ph_w64 : (void*)Lc.d_ph_w32),
        (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)Lc.d_out,
        (V*)Lp.d_out);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  // translation at every level
  for (int s = 0; s < c->nlev; ++s) {
    Level& L = c->lev[s];
    int nchunk = (L.K + kc - 1) / kc;
    pbeg(c, st, "translate", s,
         2.0 * L.nbox * L.K * 4 * R_ * es + (double)L.off_dx.size() * L.K * es,
         8.0 * L.il_src.size() * L.K * 4 * R_);
    k_translate<T><<<(unsigned)(L.nbox * nchunk), 256, 0, st>>>(
        L.nbox, L.K, R, kc, L.d_il_ptr, L.d_il_src, L.d_il_off,
        (const V*)(f64 ? (void*)L.d_T64 : (void*)L.d_T32), (const V*)L.d_out, (V*)L.d_in);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  // downward
  for (int s = c->nlev - 2; s >= 0; --s) {
    Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
    int nchunk = (Lc.K + kc - 1) / kc;
    pbeg(c, st, "anterpolate", s,
         ((double)Lp.nbox * Lp.K + 2.0 * Lc.nbox * Lc.K) * 4 * R_ * es +
             (double)Lc.ant_nnz * (4.0 + es / 2) + 4.0 * Lp.K * es,
         (double)Lc.nbox * Lc.ant_nnz * (34.0 * R_));
    k_anterp<T><<<(unsigned)(Lc.nbox * nchunk), 256, 0, st>>>(
        Lc.nbox, Lc.K, Lp.K, R, kc, Lc.d_parent, Lc.d_quad, Lc.d_ant_ptr, Lc.d_ant_idx,
        (const T*)(f64 ? (void*)Lc.d_ant_w64 : (void*)Lc.d_ant_w32),
        (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)Lp.d_in,
        (V*)Lc.d_in);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  // receive
  {
    int rc = std::min(R, std::max(1, 256 / c->npsi));
    rc = std::min(rc, 4);
    int nrc = (R + rc - 1) / rc;
    size_t sm = (size_t)L0.K * 4 * rc * sizeof(V);
    cudaFuncSetAttribute(k_receive<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    pbeg(c, st, "receive", 0,
         (double)c->p * L0.K * 4 * R_ * es + (double)c->S * c->npsi * 2 * L0.K * es +
             (accumulate ? 2.0 : 1.0) * c->p * 2 * c->npsi * R_ * 16,
         48.0 * c->p * c->npsi * L0.K * R_);
    k_receive<T><<<(unsigned)(c->p * nrc), c->npsi * rc, sm, st>>>(
        c->p, L0.K, c->npsi, R, rc, nrc, (const V*)L0.d_in,
        (const V*)(f64 ? (void*)c->d_P64 : (void*)c->d_P32), c->d_sid, L0.d_w, c->d_dshift,
        c->any_dshift, L0.d_khat, c->k, c->zeta, y, accumulate ? 1 : 0);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  return SMR_OK;
}

int run_far(Ctx* c, int R, int prec, const double2* x, double2* y, bool accumulate,
            cudaStream_t st) {
  int rc = ensure_spectra(c, R, prec);
  if (rc) return rc;
  return prec == SMR_PREC_FP64 ? far_impl<double>(c, R, x, y, accumulate, st)
                               : far_impl<float>(c, R, x, y, accumulate, st);
}

template <typename T>
static int bs_impl(Ctx* c, int nrow, int R, const int* ptr, const int* col, const int* blk,
                   const void* Bt, const double2* x, double2* y, bool acc, cudaStream_t st) {
  typedef typename CV<T>::V V;
  int n2 = 2 * c->npsi;
  int rc = std::min(R, std::max(1, 256 / n2));
  int nrc = (R + rc - 1) / rc;
  size_t sm = (size_t)n2 * rc * sizeof(V);
  k_blocksparse<T><<<(unsigned)(nrow * nrc), n2 * rc, sm, st>>>(nrow, n2, R, rc, nrc, ptr, col, blk,
                                                               (const V*)Bt, x, y, acc ? 1 : 0);
  SMR_LAUNCH(c);
  return SMR_OK;
}

int run_near(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st) {
  double n2 = 2.0 * c->npsi, es = prec == SMR_PREC_FP64 ? 16 : 8;
  pbeg(c, st, "near", -1, 2.0 * c->p * n2 * R * 16 + (double)c->nblk * n2 * n2 * es,
       8.0 * n2 * n2 * c->nr_col.size() * R);
  int rc = (prec == SMR_PREC_FP64)
               ? bs_impl<double>(c, c->p, R, c->d_nr_ptr, c->d_nr_col, c->d_nr_blk, c->d_B64, x, y, false, st)
               : bs_impl<float>(c, c->p, R, c->d_nr_ptr, c->d_nr_col, c->d_nr_blk, c->d_B32, x, y, false, st);
  pend(c, st);
  return rc;
}

int run_precond(Ctx* c, int R, int prec, const double2* r, double2* z, cudaStream_t st) {
  if (prec == SMR_PREC_FP64)
    return bs_impl<double>(c, c->p, R, c->d_pc_ptr, c->d_pc_col, c->d_pc_blk, c->d_Pinv64, r, z, false, st);
  return bs_impl<float>(c, c->p, R, c->d_pc_ptr, c->d_pc_col, c->d_pc_blk, c->d_Pinv32, r, z, false, st);
}

}  // namespace smr
