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
__device__ __forceinline__ float2 cvt2(float2 v, float2) { return v; }
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

// the 4 fields of one direction (single right-hand side): 32 or 64 bytes
__device__ __forceinline__ void ld_dir(const float2* p, float2* v) {
  float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void ld_dir(const double2* p, double2* v) {
  v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
}
__device__ __forceinline__ void st_dir(float2* p, const float2* v) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}
__device__ __forceinline__ void st_dir(double2* p, const double2* v) {
  p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = v[3];
}


// ------------------------------------------------------------------ 16-byte direction parts
// Single right-hand side kernels give each thread one 16-byte part of a
// direction's 4 fields (FP32: 2 fields as a float4, FP64: 1 field), so that
// a warp instruction reads or writes one contiguous 512-byte run and shared
// memory is accessed without bank conflicts.  NT threads share a direction.
template <typename T> struct Part;
template <> struct Part<float> {
  typedef float4 H;
  static constexpr int NT = 2, FPT = 2;
  static __device__ __forceinline__ H zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void rfma(H& a, float w, H v) {
    a.x = fmaf(w, v.x, a.x); a.y = fmaf(w, v.y, a.y); a.z = fmaf(w, v.z, a.z); a.w = fmaf(w, v.w, a.w);
  }
  // a += s * v for each complex field of v
  static __device__ __forceinline__ void cfma(H& a, float2 s, H v) {
    a.x = fmaf(s.x, v.x, a.x); a.x = fmaf(-s.y, v.y, a.x);
    a.y = fmaf(s.x, v.y, a.y); a.y = fmaf(s.y, v.x, a.y);
    a.z = fmaf(s.x, v.z, a.z); a.z = fmaf(-s.y, v.w, a.z);
    a.w = fmaf(s.x, v.w, a.w); a.w = fmaf(s.y, v.z, a.w);
  }
  static __device__ __forceinline__ void add(H& a, H v) { a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w; }
  static __device__ __forceinline__ void w4(const float* p, float* w) {
    float4 a = *reinterpret_cast<const float4*>(p);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  }
};
template <> struct Part<double> {
  typedef double2 H;
  static constexpr int NT = 4, FPT = 1;
  static __device__ __forceinline__ H zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void rfma(H& a, double w, H v) { a.x = fma(w, v.x, a.x); a.y = fma(w, v.y, a.y); }
  static __device__ __forceinline__ void cfma(H& a, double2 s, H v) {
    a.x = fma(s.x, v.x, a.x); a.x = fma(-s.y, v.y, a.x);
    a.y = fma(s.x, v.y, a.y); a.y = fma(s.y, v.x, a.y);
  }
  static __device__ __forceinline__ void add(H& a, H v) { a.x += v.x; a.y += v.y; }
  static __device__ __forceinline__ void w4(const double* p, double* w) {
    double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
  }
};
template <typename T>
__device__ __forceinline__ typename Part<T>::H ldp(const typename CV<T>::V* base, size_t dir, int h) {
  return reinterpret_cast<const typename Part<T>::H*>(base + dir * 4)[h];
}
template <typename T>
__device__ __forceinline__ void stp(typename CV<T>::V* base, size_t dir, int h, typename Part<T>::H v) {
  reinterpret_cast<typename Part<T>::H*>(base + dir * 4)[h] = v;
}

// ------------------------------------------------------------------ aggregation
// out0[mu][k][f][r] = shift * sum_n conj(P[s][n][comp f][k]) x[mu][cur f][n][r]
// One CTA = a tile of up to 16 particles of one shape (x in shared memory) x a
// chunk of 64 directions; each pattern value is reused for the tile's columns.
template <typename T>
__global__ void k_aggregate(int K0, int npsi, int R, int RC, int nkc,
                            const int* __restrict__ tile_shape, const int* __restrict__ tile_start,
                            const int* __restrict__ tile_count, const int* __restrict__ perm,
                            const double2* __restrict__ x, const typename CV<T>::V* __restrict__ P,
                            const double* __restrict__ dshift, int any_dshift,
                            const double* __restrict__ khat, double k,
                            typename CV<T>::V* __restrict__ out) {
  typedef typename CV<T>::V V;
  extern __shared__ unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);          // [col][2][npsi]
  int nrc = (R + RC - 1) / RC;
  int TP = max(1, 16 / RC);                        // particles per column group
  int nsub = (16 + TP - 1) / TP;
  int tile = blockIdx.x / (nsub * nkc * nrc);
  int rest = blockIdx.x % (nsub * nkc * nrc);
  int sub = rest / (nkc * nrc);
  rest %= nkc * nrc;
  int kc = rest / nrc, r0 = (rest % nrc) * RC;
  int nr = min(RC, R - r0);
  int s = tile_shape[tile], tp = tile_count[tile];
  int t0 = tile_start[tile] + sub * TP;
  int np_ = min(tp - sub * TP, TP);
  if (np_ <= 0) return;
  int ncol = np_ * nr;
  // stage x for the tile's columns (particle, r)
  for (int t = threadIdx.x; t < ncol * 2 * npsi; t += blockDim.x) {
    int n = t % npsi, cc = (t / npsi) % 2, col = t / (2 * npsi);
    int mu = perm[t0 + col / nr], r = r0 + col % nr;
    xs[(col * 2 + cc) * npsi + n] = cvt2(x[((size_t)mu * 2 * npsi + cc * npsi + n) * R + r], V());
  }
  __syncthreads();
  int kl = threadIdx.x & 63, g = threadIdx.x >> 6;   // 64 directions x 4 column groups
  int kk = kc * 64 + kl;
  if (kk >= K0) return;
  const V* Ps = P + (size_t)s * npsi * 2 * K0 + kk;
  V acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[q][f] = czero<V>();
  for (int n = 0; n < npsi; ++n) {
    V pt = Ps[(size_t)(2 * n) * K0], pp = Ps[(size_t)(2 * n + 1) * K0];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int col = g + 4 * q;
      if (col < ncol) {
        V e = xs[(col * 2) * npsi + n], m = xs[(col * 2 + 1) * npsi + n];
        cfmac(acc[q][0], pt, e);
        cfmac(acc[q][1], pp, e);
        cfmac(acc[q][2], pt, m);
        cfmac(acc[q][3], pp, m);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int col = g + 4 * q;
    if (col >= ncol) continue;
    int mu = perm[t0 + col / nr], r = r0 + col % nr;
    if (any_dshift) {
      const double* d = dshift + 3 * mu;
      const double* kh = khat + 3 * kk;
      double ph = k * (kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2]);
      double sn, cs;
      sincos(ph, &sn, &cs);
      V sh = mkc((T)cs, (T)sn);
      for (int f = 0; f < 4; ++f) acc[q][f] = cmul(acc[q][f], sh);
    }
    V* o = out + ((size_t)mu * K0 + kk) * 4 * R + r;
    o[0] = acc[q][0]; o[R] = acc[q][1]; o[2 * R] = acc[q][2]; o[3 * R] = acc[q][3];
  }
}

// ------------------------------------------------------------------ interpolation (separable)
// One warp per row of the output grid; lanes stride over (column, field, r).
// R1 = (R == 1) lets the compiler turn the column / field split into shifts.
template <bool R1>
__device__ __forceinline__ void split_e(int e, int R4, int* j, int* fr) {
  if (R1) { *j = e >> 2; *fr = e & 3; }
  else { *j = e / R4; *fr = e - *j * R4; }
}

// theta pass:  G[c][tp][j][f][r] = sum_a w_a sgn_a F[c][row_a][(j + refl_a N/2) mod N][f][r]
template <typename T, bool R1>
__global__ void k_interp_theta(int nrows, int nthP, int nphC, int Kc, int R,
                               const int* __restrict__ th_src, const int* __restrict__ th_refl,
                               const T* __restrict__ th_w, const typename CV<T>::V* __restrict__ F,
                               typename CV<T>::V* __restrict__ G) {
  typedef typename CV<T>::V V;
  int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nrows) return;
  int c = row / nthP, tp = row - c * nthP;
  int R4 = 4 * R;
  int srow[4];
  T w[4];
  bool rf[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    rf[a] = th_refl[tp * 4 + a] != 0;
    w[a] = rf[a] ? -th_w[tp * 4 + a] : th_w[tp * 4 + a];
    srow[a] = th_src[tp * 4 + a] * nphC;
  }
  const V* src = F + (size_t)c * Kc * R4;
  V* dst = G + (size_t)row * nphC * R4;
  int half = nphC >> 1, n = nphC * R4;
  for (int e = lane; e < n; e += 32) {
    int j, fr;
    split_e<R1>(e, R4, &j, &fr);
    int jr = j + half;
    jr = jr >= nphC ? jr - nphC : jr;
    V acc = czero<V>();
#pragma unroll
    for (int a = 0; a < 4; ++a) rfma(acc, w[a], src[(size_t)(srow[a] + (rf[a] ? jr : j)) * R4 + fr]);
    dst[e] = acc;
  }
}

// phi pass, shift and child sum:
//   out[B][tp][jp][f][r] = sum_c shift[q_c][tp, jp] sum_b w_b G[c][tp][col_b][f][r]
template <typename T, bool R1>
__global__ void k_interp_phi(int nrows, int nthP, int nphP, int nphC, int R,
                             const int* __restrict__ ch_ptr, const int* __restrict__ ch_idx,
                             const int* __restrict__ ch_quad, const int* __restrict__ ph_src,
                             const T* __restrict__ ph_w, const typename CV<T>::V* __restrict__ shift,
                             const typename CV<T>::V* __restrict__ G,
                             typename CV<T>::V* __restrict__ out) {
  typedef typename CV<T>::V V;
  int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nrows) return;
  int B = row / nthP, tp = row - B * nthP;
  int Kp = nthP * nphP, R4 = 4 * R;
  int e0 = ch_ptr[B], e1 = ch_ptr[B + 1];
  const V* gch[4];
  const V* sh[4];
  int nch = e1 - e0;
  for (int q = 0; q < nch; ++q) {
    gch[q] = G + ((size_t)ch_idx[e0 + q] * nthP + tp) * nphC * R4;
    sh[q] = shift + (size_t)ch_quad[e0 + q] * Kp + (size_t)tp * nphP;
  }
  V* dst = out + (size_t)row * nphP * R4;
  int n = nphP * R4;
  for (int e = lane; e < n; e += 32) {
    int jp, fr;
    split_e<R1>(e, R4, &jp, &fr);
    int col[4];
    T w[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) { col[b] = ph_src[jp * 4 + b] * R4 + fr; w[b] = ph_w[jp * 4 + b]; }
    V acc = czero<V>();
    for (int q = 0; q < nch; ++q) {
      V tsum = czero<V>();
#pragma unroll
      for (int b = 0; b < 4; ++b) rfma(tsum, w[b], gch[q][col[b]]);
      cfma(acc, sh[q][jp], tsum);
    }
    dst[e] = acc;
  }
}

// Fused interpolation: per parent box and tile of TR parent rows, each child's
// theta pass goes to shared memory and the phi pass, shift and child sum are
// accumulated in registers (at most EMAX outputs per thread).
constexpr int EMAX = 12;
template <typename T, bool R1>
__global__ void k_interp_fused(int nthP, int nphP, int nphC, int Kc, int R, int TR, int nrt,
                               const int* __restrict__ ch_ptr, const int* __restrict__ ch_idx,
                               const int* __restrict__ ch_quad, const int* __restrict__ th_src,
                               const int* __restrict__ th_refl, const T* __restrict__ th_w,
                               const int* __restrict__ ph_src, const T* __restrict__ ph_w,
                               const typename CV<T>::V* __restrict__ shift,
                               const typename CV<T>::V* __restrict__ F, typename CV<T>::V* __restrict__ out) {
  typedef typename CV<T>::V V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* G = reinterpret_cast<V*>(smem_raw);           // [TR][nphC][4R]
  int B = blockIdx.x / nrt, rt = blockIdx.x % nrt;
  int tp0 = rt * TR, ntr = min(TR, nthP - tp0);
  int R4 = 4 * R, Kp = nthP * nphP;
  int rowG = nphC * R4, rowP = nphP * R4;
  int nG = ntr * rowG, nel = ntr * rowP;
  int half = nphC >> 1;
  V acc[EMAX];
#pragma unroll
  for (int i = 0; i < EMAX; ++i) acc[i] = czero<V>();
  for (int e = ch_ptr[B]; e < ch_ptr[B + 1]; ++e) {
    const V* src = F + (size_t)ch_idx[e] * Kc * R4;
    const V* sh = shift + (size_t)ch_quad[e] * Kp + (size_t)tp0 * nphP;
    __syncthreads();
    for (int t = threadIdx.x; t < nG; t += blockDim.x) {
      int tr = t / rowG, rem = t - tr * rowG;
      int j, fr;
      split_e<R1>(rem, R4, &j, &fr);
      int tp = tp0 + tr;
      int jr = j + half;
      jr = jr >= nphC ? jr - nphC : jr;
      V a = czero<V>();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int refl = th_refl[tp * 4 + q];
        T w = refl ? -th_w[tp * 4 + q] : th_w[tp * 4 + q];
        rfma(a, w, src[(size_t)(th_src[tp * 4 + q] * nphC + (refl ? jr : j)) * R4 + fr]);
      }
      G[t] = a;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < EMAX; ++i) {
      int t = threadIdx.x + i * blockDim.x;
      if (t < nel) {
        int tr = t / rowP, rem = t - tr * rowP;
        int jp, fr;
        split_e<R1>(rem, R4, &jp, &fr);
        const V* g = G + tr * rowG + fr;
        V sum = czero<V>();
#pragma unroll
        for (int b = 0; b < 4; ++b) rfma(sum, ph_w[jp * 4 + b], g[ph_src[jp * 4 + b] * R4]);
        cfma(acc[i], sh[tr * nphP + jp], sum);
      }
    }
  }
  V* dst = out + ((size_t)B * Kp + (size_t)tp0 * nphP) * R4;
#pragma unroll
  for (int i = 0; i < EMAX; ++i) {
    int t = threadIdx.x + i * blockDim.x;
    if (t < nel) dst[t] = acc[i];
  }
}


// Single right-hand side: CTA = (parent box, tile of TR parent theta rows);
// each thread owns up to EM1 parent direction parts of the tile across the
// loop over the children.  Per child: theta pass of the tile's rows into
// shared memory G[TR][nphC][4] (4 taps, tables read as 16-byte vectors), then
// phi pass, shift and child sum in registers.
template <typename T> struct EM1 { static constexpr int v = sizeof(T) == 4 ? 8 : 12; };
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_interp1(int nthP, int nphP, unsigned mP, int nphC, int Kc, int TR, int nrt,
                                                 const int* __restrict__ ch_ptr, const int* __restrict__ ch_idx,
                                                 const int* __restrict__ ch_quad, const int* __restrict__ th_pk,
                                                 const T* __restrict__ th_w,
                                                 const int* __restrict__ ph_src, const T* __restrict__ ph_w,
                                                 const typename CV<T>::V* __restrict__ shift,
                                                 const typename CV<T>::V* __restrict__ F,
                                                 typename CV<T>::V* __restrict__ out) {
  typedef typename CV<T>::V V;
  typedef Part<T> P;
  typedef typename P::H H;
  constexpr int NT = P::NT, EM = EM1<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* G = reinterpret_cast<V*>(smem_raw);           // [TR][nphC][4]
  int B = blockIdx.x / nrt, rt = blockIdx.x - (blockIdx.x / nrt) * nrt;
  int tp0 = rt * TR, ntr = min(TR, nthP - tp0);
  int Kp = nthP * nphP;
  int nout = ntr * nphP * NT;
  int half = nphC >> 1;
  // (row, column) of this thread's tasks, stepped by the NTH tasks of one
  // sweep of the CTA without dividing per task
  const int NTH = blockDim.x / NT, task0 = threadIdx.x / NT, h = threadIdx.x % NT;
  const int trG0 = task0 / nphC, jG0 = task0 - trG0 * nphC;
  const int dqG = NTH / nphC, drG = NTH - dqG * nphC;
  H acc[EM];
#pragma unroll
  for (int i = 0; i < EM; ++i) acc[i] = P::zero();
  for (int e = ch_ptr[B]; e < ch_ptr[B + 1]; ++e) {
    const V* src = F + (size_t)ch_idx[e] * Kc * 4;
    const V* sh = shift + (size_t)ch_quad[e] * Kp + (size_t)tp0 * nphP;
    __syncthreads();
    for (int tr = trG0, j = jG0, task = task0; tr < ntr; task += NTH) {
      int tp = tp0 + tr;
      int jr = j + half;
      jr = jr >= nphC ? jr - nphC : jr;
      int4 pk = *reinterpret_cast<const int4*>(th_pk + tp * 4);
      T w[4];
      P::w4(th_w + tp * 4, w);
      H a = P::zero();
      P::rfma(a, w[0], ldp<T>(src, (size_t)(pk.x & 0xffff) * nphC + ((pk.x >> 16) ? jr : j), h));
      P::rfma(a, w[1], ldp<T>(src, (size_t)(pk.y & 0xffff) * nphC + ((pk.y >> 16) ? jr : j), h));
      P::rfma(a, w[2], ldp<T>(src, (size_t)(pk.z & 0xffff) * nphC + ((pk.z >> 16) ? jr : j), h));
      P::rfma(a, w[3], ldp<T>(src, (size_t)(pk.w & 0xffff) * nphC + ((pk.w >> 16) ? jr : j), h));
      stp<T>(G, task, h, a);
      j += drG;
      tr += dqG;
      if (j >= nphC) { j -= nphC; ++tr; }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < EM; ++i) {
      // task / nphP as a multiply-high by ceil(2^32 / nphP): exact while task * nphP < 2^32
      const unsigned task = (unsigned)(task0 + i * NTH);
      const int tr = (int)__umulhi(task, mP), jp = (int)task - tr * nphP;
      if (tr < ntr) {
        int4 cs = *reinterpret_cast<const int4*>(ph_src + jp * 4);
        T w[4];
        P::w4(ph_w + jp * 4, w);
        size_t rb = (size_t)tr * nphC;
        H sm = P::zero();
        P::rfma(sm, w[0], ldp<T>(G, rb + cs.x, h));
        P::rfma(sm, w[1], ldp<T>(G, rb + cs.y, h));
        P::rfma(sm, w[2], ldp<T>(G, rb + cs.z, h));
        P::rfma(sm, w[3], ldp<T>(G, rb + cs.w, h));
        P::cfma(acc[i], sh[tr * nphP + jp], sm);
      }
    }
  }
  V* dst = out + ((size_t)B * Kp + (size_t)tp0 * nphP) * 4;
#pragma unroll
  for (int i = 0; i < EM; ++i) {
    int t = threadIdx.x + i * blockDim.x;
    if (t < nout) stp<T>(dst, t / NT, t % NT, acc[i]);
  }
}
// ------------------------------------------------------------------ translation
// in[b][k] = sum_{(b', o) in IL(b)} T[o][k] out[b'][k]   (Eqs. 22-23)
// One CTA = 4x4 target boxes of the lattice x a chunk of directions; the 8x8
// source halo and the table rows of the chunk are staged in shared memory,
// so each source spectrum is fetched about 4 times instead of 27.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// 4 consecutive complex values (the 4 fields of one direction) from shared memory
__device__ __forceinline__ void load4(const float2* p, float2* v) {
  float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2* v) {
  v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
}

template <typename T>
__global__ void k_translate(int K, int R, int RC, int KC, int ntx, int ntile, const int* __restrict__ tiles,
                            int map_x0, int map_y0, int map_w, int map_h, int noff,
                            const int* __restrict__ boxmap,
                            const int* __restrict__ offid, const typename CV<T>::V* __restrict__ Tt,
                            const typename CV<T>::V* __restrict__ out,
                            typename CV<T>::V* __restrict__ in) {
  typedef typename CV<T>::V V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int nrc = (R + RC - 1) / RC;
  int tile = tiles[blockIdx.x % ntile];
  int rest = blockIdx.x / ntile;
  int rch = rest % nrc, kch = rest / nrc;
  int tx = tile % ntx, ty = tile / ntx;
  // absolute lattice origin of the tile, aligned to multiples of 4
  int ax0 = ((map_x0 >> 2) + tx) * 4, ay0 = ((map_y0 >> 2) + ty) * 4;
  int k0 = kch * KC, r0 = rch * RC;
  int nk = min(KC, K - k0), nr = min(RC, R - r0);
  int W = KC * 4 * RC;                                // V per source box in the chunk
  V* S = reinterpret_cast<V*>(smem_raw);              // [64 sources][KC][4][RC]
  V* Ts = S + 64 * W;                                 // [noff][KC]
  int* bid = reinterpret_cast<int*>(Ts + max(noff, 1) * KC);   // [64] source box ids
  int* tgt = bid + 64;                                // [16] target box ids
  int* cnt = tgt + 16;                                // [16] candidate counts
  int2* lst = reinterpret_cast<int2*>(cnt + 16);      // [16][27] (source slot, table row)
  for (int t = threadIdx.x; t < 64; t += blockDim.x) {
    int sx = ax0 - 2 + (t & 7), sy = ay0 - 2 + (t >> 3);
    int lx = sx - map_x0, ly = sy - map_y0;
    bid[t] = (lx >= 0 && ly >= 0 && lx < map_w && ly < map_h) ? boxmap[ly * map_w + lx] : -1;
  }
  __syncthreads();
  if (RC == R) {
    // each source box's chunk is contiguous in global memory: asynchronous
    // 16-byte copies, zero-filled for missing boxes and past the last direction
    int per = W * (int)sizeof(V) / 16;
    int valid = nk * 4 * R * (int)sizeof(V);
    for (int t = threadIdx.x; t < 64 * per; t += blockDim.x) {
      int sb = t / per, pc = t - sb * per;
      int b = bid[sb];
      const char* g = reinterpret_cast<const char*>(out);
      int nb = 0;
      if (b >= 0 && pc * 16 < valid) {
        g += ((size_t)b * K + k0) * 4 * R * sizeof(V) + (size_t)pc * 16;
        nb = 16;
      }
      cp_async16(reinterpret_cast<char*>(S + (size_t)sb * W) + pc * 16, g, nb);
    }
  } else if ((R * (int)sizeof(V)) % 16 == 0 && (RC * (int)sizeof(V)) % 16 == 0) {
    // asynchronous 16-byte copies of each (source, direction, field) run of RC
    // columns (aligned: R and RC span whole 16-byte pieces), zero-filled for
    // missing boxes, past the last direction and past the last column
    int pr = RC * (int)sizeof(V) / 16;               // pieces per run
    int per = KC * 4 * pr;                           // pieces per source box
    for (int t = threadIdx.x; t < 64 * per; t += blockDim.x) {
      int sb = t / per, e = t - sb * per;
      int run = e / pr, pc = e - run * pr;           // run = kl * 4 + f
      int kl = run >> 2;
      int b = bid[sb];
      const char* g = reinterpret_cast<const char*>(out);
      int nb = 0;
      int col = pc * 16 / (int)sizeof(V);            // first column of the piece
      if (b >= 0 && kl < nk && col < nr) {
        g += ((((size_t)b * K + k0 + kl) * 4 + (run & 3)) * R + r0) * sizeof(V) + (size_t)pc * 16;
        nb = 16;
      }
      cp_async16(reinterpret_cast<char*>(S + (size_t)sb * W + (size_t)run * RC) + pc * 16, g, nb);
    }
  } else {
    for (int t = threadIdx.x; t < 64 * W; t += blockDim.x) {
      int sb = t / W, e = t % W;
      int rl = e % RC, kl = e / (4 * RC), f = (e / RC) % 4;
      int b = bid[sb];
      S[t] = (b >= 0 && kl < nk && rl < nr) ? out[(((size_t)b * K + k0 + kl) * 4 + f) * R + r0 + rl]
                                           : czero<V>();
    }
  }
  for (int t = threadIdx.x; t < noff * KC; t += blockDim.x) {
    int o = t / KC, kl = t % KC;
    Ts[t] = (kl < nk) ? Tt[(size_t)o * K + k0 + kl] : czero<V>();
  }
  if (threadIdx.x < 16) {
    int tg = threadIdx.x;
    int ix = ax0 + (tg & 3), iy = ay0 + (tg >> 2);
    int lx = ix - map_x0, ly = iy - map_y0;
    int b = (lx >= 0 && ly >= 0 && lx < map_w && ly < map_h) ? boxmap[ly * map_w + lx] : -1;
    tgt[tg] = b;
    int n = 0;
    if (b >= 0) {
      int px = ix >> 1, py = iy >> 1;
      for (int cy = 2 * py - 2; cy <= 2 * py + 3; ++cy)
        for (int cx = 2 * px - 2; cx <= 2 * px + 3; ++cx) {
          int dx = ix - cx, dy = iy - cy;
          if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
          int sb = (cy - ay0 + 2) * 8 + (cx - ax0 + 2);
          int o = offid[(dx + 3) * 7 + (dy + 3)];
          if (bid[sb] < 0 || o < 0 || n >= 27) continue;
          lst[tg * 27 + n] = make_int2(sb * W, o * KC);
          ++n;
        }
    }
    cnt[tg] = n;
  }
  cp_async_wait_all();
  __syncthreads();
  // outputs: 16 targets x nk directions x nr columns, 4 fields each
  int nout = 16 * nk * nr;
  for (int t = threadIdx.x; t < nout; t += blockDim.x) {
    int rl = t % nr, kl = (t / nr) % nk, tg = t / (nr * nk);
    int b = tgt[tg];
    if (b < 0) continue;
    V acc[4] = {czero<V>(), czero<V>(), czero<V>(), czero<V>()};
    int n = cnt[tg];
    const int2* L = lst + tg * 27;
    int kr = kl * 4 * RC + rl;
    for (int e = 0; e < n; ++e) {
      int2 so = L[e];
      V tv = Ts[so.y + kl];
      const V* sv = S + so.x + kr;
      V v[4];
      if (RC == 1) {
        load4(sv, v);
      } else {
        v[0] = sv[0]; v[1] = sv[RC]; v[2] = sv[2 * RC]; v[3] = sv[3 * RC];
      }
      cfma(acc[0], tv, v[0]);
      cfma(acc[1], tv, v[1]);
      cfma(acc[2], tv, v[2]);
      cfma(acc[3], tv, v[3]);
    }
    V* o = in + ((size_t)b * K + k0 + kl) * 4 * R + r0 + rl;
    for (int f = 0; f < 4; ++f) o[f * R] = acc[f];
  }
}

// Single right-hand side: each thread owns one 16-byte part of the 2x2
// targets that share one parent, for one direction, and walks the parent's
// 6x6 source window once; a staged source part is read from shared memory
// once for all four targets (conflict-free: lanes read consecutive 16-byte
// parts).  CTA = 8x8 targets (4x4 parents) x KC directions; 16 x KC x NT threads.
template <typename T, int KC>
__global__ void __launch_bounds__(512, 2) k_translate1(int K, int ntx, int ntile,
                                                    const int* __restrict__ tiles, int map_x0, int map_y0,
                                                    int map_w, int map_h, const int* __restrict__ boxmap,
                                                    const typename CV<T>::V* __restrict__ Tg,
                                                    const typename CV<T>::V* __restrict__ out,
                                                    typename CV<T>::V* __restrict__ in) {
  typedef typename CV<T>::V V;
  typedef Part<T> P;
  typedef typename P::H H;
  constexpr int NT = P::NT;
  constexpr int TS = 8, HS = TS + 4;                  // targets per side, halo per side
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int tile = tiles[blockIdx.x % ntile];
  int kch = blockIdx.x / ntile;
  int tx = tile % ntx, ty = tile / ntx;
  int ax0 = ((map_x0 >> 3) + tx) * TS, ay0 = ((map_y0 >> 3) + ty) * TS;
  int k0 = kch * KC;
  int nk = min(KC, K - k0);
  constexpr int W = KC * 4;
  V* S = reinterpret_cast<V*>(smem_raw);              // [HS*HS sources][KC][4]
  V* Ts = S + HS * HS * W;                            // [49 offsets][KC]
  // FP32: the table entries as (t_r, t_r, -t_i, t_i), so that a complex
  // multiply-add of two fields is four packed FMAs
  constexpr bool PK = sizeof(T) == 4;
  float4* Ts4 = reinterpret_cast<float4*>(Ts);
  int* bid = reinterpret_cast<int*>(PK ? reinterpret_cast<unsigned char*>(Ts4 + 49 * KC)
                                       : reinterpret_cast<unsigned char*>(Ts + 49 * KC));   // [HS*HS] source box ids
  int* tb = bid + HS * HS;                            // [TS*TS] target box ids
  for (int t = threadIdx.x; t < HS * HS + TS * TS; t += blockDim.x) {
    int sx, sy;
    if (t < HS * HS) { sx = ax0 - 2 + t % HS; sy = ay0 - 2 + t / HS; }
    else { int u = t - HS * HS; sx = ax0 + u % TS; sy = ay0 + u / TS; }
    int lx = sx - map_x0, ly = sy - map_y0;
    bid[t] = (lx >= 0 && ly >= 0 && lx < map_w && ly < map_h) ? boxmap[ly * map_w + lx] : -1;
  }
  __syncthreads();
  {
    constexpr int per = W * (int)sizeof(V) / 16;      // 16-byte pieces per source row
    int valid = nk * 4 * (int)sizeof(V);
    for (int t = threadIdx.x; t < HS * HS * per; t += blockDim.x) {
      int sb = t / per, pc = t - sb * per;
      int b = bid[sb];
      const char* g = reinterpret_cast<const char*>(out);
      int nb = 0;
      if (b >= 0 && pc * 16 < valid) {
        g += ((size_t)b * K + k0) * 4 * sizeof(V) + (size_t)pc * 16;
        nb = 16;
      }
      cp_async16(reinterpret_cast<char*>(S + (size_t)sb * W) + pc * 16, g, nb);
    }
  }
  for (int t = threadIdx.x; t < 49 * KC; t += blockDim.x) {
    int o = t / KC, kl = t - o * KC;
    const V tv = (kl < nk) ? Tg[(size_t)o * K + k0 + kl] : czero<V>();
    if constexpr (PK) Ts4[t] = make_float4((float)tv.x, (float)tv.x, -(float)tv.y, (float)tv.y);
    else Ts[t] = tv;
  }
  cp_async_wait_all();
  __syncthreads();
  const int h = threadIdx.x % NT;
  const int kl = (threadIdx.x / NT) % KC, par = threadIdx.x / (NT * KC);   // parent 0..15 of the tile
  if (kl >= nk || par >= (TS / 2) * (TS / 2)) return;
  int pxo = (par % (TS / 2)) * 2, pyo = (par / (TS / 2)) * 2;
  bool any = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) any |= tb[(pyo + (q >> 1)) * TS + (pxo + (q & 1))] >= 0;
  if (!any) return;
  const V* Sp = S + (size_t)(pyo * HS + pxo) * W + kl * 4;   // window origin
  const V* Tp = Ts + kl;
  H acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = P::zero();
  // the parent's 6x6 source window; target q = (q & 1, q >> 1) inside the
  // parent; offset (dx, dy) = target - source is known at compile time
#pragma unroll
  for (int wy = 0; wy < 6; ++wy) {
#pragma unroll
    for (int wx = 0; wx < 6; ++wx) {
      H v = reinterpret_cast<const H*>(Sp + (wy * HS + wx) * W)[h];
      if constexpr (PK) {
        // (re, im) += (t_r, t_r) (v_re, v_im) + (-t_i, t_i) (v_im, v_re), per field
        const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
        const float2 s0 = make_float2(v.y, v.x), s1 = make_float2(v.w, v.z);
        const float4* T4 = Ts4 + kl;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int dx = (q & 1) + 2 - wx, dy = (q >> 1) + 2 - wy;
          if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
          const float4 t = T4[((dx + 3) * 7 + (dy + 3)) * KC];
          const float2 tr = make_float2(t.x, t.y), tn = make_float2(t.z, t.w);
          float2 a0 = make_float2(acc[q].x, acc[q].y), a1 = make_float2(acc[q].z, acc[q].w);
          a0 = __ffma2_rn(tr, v0, a0);
          a0 = __ffma2_rn(tn, s0, a0);
          a1 = __ffma2_rn(tr, v1, a1);
          a1 = __ffma2_rn(tn, s1, a1);
          acc[q] = make_float4(a0.x, a0.y, a1.x, a1.y);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int dx = (q & 1) + 2 - wx, dy = (q >> 1) + 2 - wy;
          if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
          P::cfma(acc[q], Tp[((dx + 3) * 7 + (dy + 3)) * KC], v);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int b = tb[(pyo + (q >> 1)) * TS + (pxo + (q & 1))];
    if (b < 0) continue;
    stp<T>(in, (size_t)b * K + k0 + kl, h, acc[q]);
  }
}

// Few boxes, many directions (coarse levels), one right-hand side: threads run
// along the directions (NT 16-byte parts each, coalesced); a CTA takes TG
// consecutive target boxes and reads each target's interaction list
// (source box * 64 + table row) uniformly.
template <typename T>
__global__ void __launch_bounds__(256) k_translate_few(int K, int nbox, int TG, const int* __restrict__ il_ptr,
                                                       const int* __restrict__ il_pk,
                                                       const typename CV<T>::V* __restrict__ Tg,
                                                       const typename CV<T>::V* __restrict__ out,
                                                       typename CV<T>::V* __restrict__ in) {
  typedef typename CV<T>::V V;
  typedef Part<T> P;
  typedef typename P::H H;
  constexpr int NT = P::NT;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int k = (int)(t / NT), h = (int)(t % NT);
  const bool ok = k < K;
  const int b0 = blockIdx.y * TG, b1 = min(nbox, b0 + TG);
  for (int b = b0; b < b1; ++b) {
    H acc = P::zero();
    for (int e = il_ptr[b]; e < il_ptr[b + 1]; ++e) {
      const int pk = il_pk[e];
      if (ok) P::cfma(acc, Tg[(size_t)(pk & 63) * K + k], ldp<T>(out, (size_t)(pk >> 6) * K + k, h));
    }
    if (ok) stp<T>(in, (size_t)b * K + k, h, acc);
  }
}

// Whole coarse level per CTA, one right-hand side: a CTA takes a chunk of
// KCH directions of every box of the level (at most a few hundred boxes),
// stages their outgoing spectra and the chunk of the 49 offset tables in
// shared memory, and computes every target's sum from there, so each source
// spectrum is read from memory once instead of once per target that lists
// it.  Tasks are (target, direction, 16-byte part), the parts of consecutive
// directions on consecutive threads.
template <typename T>
__global__ void __launch_bounds__(256) k_translate_lvl(int K, int nbox, int KCH, const int* __restrict__ il_ptr,
                                                       const int* __restrict__ il_pk,
                                                       const typename CV<T>::V* __restrict__ Tg,
                                                       const typename CV<T>::V* __restrict__ out,
                                                       typename CV<T>::V* __restrict__ in) {
  typedef typename CV<T>::V V;
  typedef Part<T> P;
  typedef typename P::H H;
  constexpr int NT = P::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* S = reinterpret_cast<V*>(smem_raw);                 // [nbox][KCH][4]
  V* Ts = S + (size_t)nbox * KCH * 4;                    // [49][KCH]
  const int k0 = blockIdx.x * KCH, kn = min(KCH, K - k0);
  // stage: every box's 4 fields for the chunk, and the tables
  for (int i = threadIdx.x; i < nbox * KCH * NT; i += blockDim.x) {
    const int b = i / (KCH * NT), r = i - b * (KCH * NT), kl = r / NT, h = r - kl * NT;
    H v = P::zero();
    if (kl < kn) v = ldp<T>(out, (size_t)b * K + k0 + kl, h);
    stp<T>(S, (size_t)b * KCH + kl, h, v);
  }
  for (int i = threadIdx.x; i < 49 * KCH; i += blockDim.x) {
    const int row = i / KCH, kl = i - row * KCH;
    Ts[i] = kl < kn ? Tg[(size_t)row * K + k0 + kl] : czero<V>();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbox * KCH * NT; i += blockDim.x) {
    const int b = i / (KCH * NT), r = i - b * (KCH * NT), kl = r / NT, h = r - kl * NT;
    if (kl >= kn) continue;
    H acc = P::zero();
    for (int e = il_ptr[b]; e < il_ptr[b + 1]; ++e) {
      const int pk = il_pk[e];
      P::cfma(acc, Ts[(pk & 63) * KCH + kl], ldp<T>(S, (size_t)(pk >> 6) * KCH + kl, h));
    }
    stp<T>(in, (size_t)b * K + k0 + kl, h, acc);
  }
}

// ------------------------------------------------------------------ anterpolation (separable adjoint)
// phi-transposed pass (one warp per row (c, tp)), child c in quadrant q of parent B:
//   Gt[c][tp][j][f][r] = w_theta_p[tp] sum_{(jp, w) in Pt(j)} w conj(shift[q][tp, jp]) in[B][tp][jp][f][r]
template <typename T, bool R1>
__global__ void k_anterp_phi(int nrows, int nthP, int nphP, int nphC, int R,
                             const int* __restrict__ parent, const int* __restrict__ quad,
                             const int* __restrict__ pht_ptr, const int* __restrict__ pht_jp,
                             const T* __restrict__ pht_w, const T* __restrict__ wthp,
                             const typename CV<T>::V* __restrict__ shift,
                             const typename CV<T>::V* __restrict__ inP,
                             typename CV<T>::V* __restrict__ Gt) {
  typedef typename CV<T>::V V;
  int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nrows) return;
  int c = row / nthP, tp = row - c * nthP;
  int Kp = nthP * nphP, R4 = 4 * R;
  const V* src = inP + ((size_t)parent[c] * Kp + (size_t)tp * nphP) * R4;
  const V* sh = shift + (size_t)quad[c] * Kp + (size_t)tp * nphP;
  T wt = wthp[tp];
  V* dst = Gt + (size_t)row * nphC * R4;
  int n = nphC * R4;
  for (int e = lane; e < n; e += 32) {
    int j, fr;
    split_e<R1>(e, R4, &j, &fr);
    V acc = czero<V>();
    for (int q = pht_ptr[j]; q < pht_ptr[j + 1]; ++q) {
      int jp = pht_jp[q];
      V sv = sh[jp];
      T w = pht_w[q] * wt;
      cfma(acc, mkc(w * sv.x, -w * sv.y), src[jp * R4 + fr]);
    }
    dst[e] = acc;
  }
}

// theta-transposed pass (one warp per child row (c, i)), sign and 1/w_theta_c folded in:
//   in[c][i][j][f][r] += sum_{(tp, w, refl) in Tt(i)} w Gt[c][tp][(j + refl N/2) mod N][f][r]
template <typename T, bool R1>
__global__ void k_anterp_theta(int nrows, int nthC, int nthP, int nphC, int R,
                               const int* __restrict__ tht_ptr, const int* __restrict__ tht_tp,
                               const int* __restrict__ tht_refl, const T* __restrict__ tht_w,
                               const typename CV<T>::V* __restrict__ Gt,
                               typename CV<T>::V* __restrict__ inC) {
  typedef typename CV<T>::V V;
  int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nrows) return;
  int c = row / nthC, i = row - c * nthC;
  int R4 = 4 * R;
  const V* g = Gt + (size_t)c * nthP * nphC * R4;
  V* dst = inC + (size_t)row * nphC * R4;
  int half = nphC >> 1, n = nphC * R4;
  int q0 = tht_ptr[i], q1 = tht_ptr[i + 1];
  for (int e = lane; e < n; e += 32) {
    int j, fr;
    split_e<R1>(e, R4, &j, &fr);
    int jr = j + half;
    jr = jr >= nphC ? jr - nphC : jr;
    V acc = czero<V>();
    for (int q = q0; q < q1; ++q)
      rfma(acc, tht_w[q], g[(size_t)(tht_tp[q] * nphC + (tht_refl[q] ? jr : j)) * R4 + fr]);
    V cur = dst[e];
    cur.x += acc.x;
    cur.y += acc.y;
    dst[e] = cur;
  }
}


// Single right-hand side, both adjoint passes fused.  CTA = (child c, tile of
// child theta rows [i0, i0 + TI), column chunk [j0, j0 + JC) of the first
// half of the phi grid together with the same chunk shifted by N/2, so that
// the pole reflection j -> j + N/2 stays inside the CTA).  The parent rows
// [lo, hi) the tile draws on get the phi-transposed pass (conjugate shift and
// parent theta weight) into shared memory; then the theta-transposed pass adds
// into the child's incoming spectrum.  Transposed taps are padded to PM / TM
// per child column / row (zero weights), packed as (tp | refl << 16).
// PMC > 0: tap tables padded to 8 per row (PM = TM = 8) and at most PMC
// real taps per row, known at compile time (tap loops unrolled)
template <typename T, int PMC>
__global__ void __launch_bounds__(256) k_anterp1(int nthC, int nphC, int nthP, int nphP, int TI, int nit,
                                                 int JC, int njc, const int* __restrict__ parent,
                                                 const int* __restrict__ quad, const int* __restrict__ lo_row,
                                                 int PM, const int* __restrict__ pjp, const T* __restrict__ pw,
                                                 const T* __restrict__ wthp,
                                                 const typename CV<T>::V* __restrict__ shift,
                                                 const typename CV<T>::V* __restrict__ inP, int TM,
                                                 const int* __restrict__ ttp, const T* __restrict__ tw,
                                                 typename CV<T>::V* __restrict__ inC) {
  typedef typename CV<T>::V V;
  typedef Part<T> P;
  typedef typename P::H H;
  constexpr int NT = P::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Gt = reinterpret_cast<V*>(smem_raw);          // [GR][2 JC][4]
  int blk = blockIdx.x;
  int jcb = blk % njc;
  blk /= njc;
  int it = blk % nit, c = blk / nit;
  int i0 = it * TI, ni = min(TI, nthC - i0);
  int half = nphC >> 1;
  int j0 = jcb * JC, nj = min(JC, half - j0);
  int lo = lo_row[it], hi = lo_row[nit + it];
  int nr = hi - lo, W = 2 * nj;
  int Kp = nthP * nphP, Kc = nthC * nphC;
  const V* srcP = inP + (size_t)parent[c] * Kp * 4;
  const V* sh = shift + (size_t)quad[c] * Kp;
  // each thread owns PPT consecutive 16-byte parts of a direction (two in
  // FP64, where a direction has four; one in FP32, where more threads hide
  // more latency); (row, column) of its tasks stepped by the NTH tasks of
  // one sweep of the CTA without dividing per task
  constexpr int PPT = sizeof(T) == 8 ? 2 : 1, NT2 = NT / PPT;
  const int NTH = blockDim.x / NT2, task0 = threadIdx.x / NT2, h = PPT * (threadIdx.x % NT2);
  const int r0 = task0 / W, u0 = task0 - r0 * W;
  const int dq = NTH / W, dr = NTH - dq * W;
  for (int r = r0, u = u0, task = task0; r < nr; task += NTH) {
    int j = (u < nj) ? j0 + u : j0 + half + (u - nj);
    int tp = lo + r;
    T wt = wthp[tp];
    const V* prow = srcP + (size_t)tp * nphP * 4;
    const V* srow = sh + (size_t)tp * nphP;
    H a = P::zero(), a1 = P::zero();
    const int pm = PMC > 0 ? 8 : PM;
#pragma unroll
    for (int q = 0; q < (PMC > 0 ? PMC : PM); q += 4) {
      int4 jj = *reinterpret_cast<const int4*>(pjp + (size_t)j * pm + q);
      T w[4];
      P::w4(pw + (size_t)j * pm + q, w);
      int js[4] = {jj.x, jj.y, jj.z, jj.w};
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (PMC > 0 && q + b >= PMC) break;
        V s = srow[js[b]];
        T ww = w[b] * wt;
        const V cw = mkc(ww * s.x, -ww * s.y);
        P::cfma(a, cw, ldp<T>(prow, js[b], h));
        if (PPT == 2) P::cfma(a1, cw, ldp<T>(prow, js[b], h + 1));
      }
    }
    stp<T>(Gt, task, h, a);
    if (PPT == 2) stp<T>(Gt, task, h + 1, a1);
    u += dr;
    r += dq;
    if (u >= W) { u -= W; ++r; }
  }
  __syncthreads();
  for (int il = r0, u = u0; il < ni;) {
    int ur = u < nj ? u + nj : u - nj;             // column j + N/2 (mod N)
    int j = (u < nj) ? j0 + u : j0 + half + (u - nj);
    int i = i0 + il;
    H a = P::zero(), a1 = P::zero();
    const int tm = PMC > 0 ? 8 : TM;
#pragma unroll
    for (int q = 0; q < (PMC > 0 ? PMC : TM); q += 4) {
      int4 pk = *reinterpret_cast<const int4*>(ttp + (size_t)i * tm + q);
      T w[4];
      P::w4(tw + (size_t)i * tm + q, w);
      int ps[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (PMC > 0 && q + b >= PMC) break;
        int r = (ps[b] & 0xffff) - lo;
        const size_t g = (size_t)r * W + ((ps[b] >> 16) ? ur : u);
        P::rfma(a, w[b], ldp<T>(Gt, g, h));
        if (PPT == 2) P::rfma(a1, w[b], ldp<T>(Gt, g, h + 1));
      }
    }
    size_t d = (size_t)c * Kc + (size_t)i * nphC + j;
    H cur = ldp<T>(inC, d, h);
    P::add(cur, a);
    stp<T>(inC, d, h, cur);
    if (PPT == 2) {
      H cur1 = ldp<T>(inC, d, h + 1);
      P::add(cur1, a1);
      stp<T>(inC, d, h + 1, cur1);
    }
    u += dr;
    il += dq;
    if (u >= W) { u -= W; ++il; }
  }
}
// FP32, one right-hand side: the anterpolation of k_anterp1 with one CTA per
// parent box serving all of its children.  Every parent tap of the
// transposed phi pass is read once and multiplied by the conjugate shifts of
// the four child quadrants (sh4: per parent direction the four quadrants'
// shifts, 32 bytes), so four accumulators share one load; the theta pass of
// each child then reads its quadrant's rows from shared memory.
template <int PMC>
__global__ void __launch_bounds__(256, 4) k_anterp4(int nthC, int nphC, int nthP, int nphP, int TI, int nit,
                                                   int JC, int njc, const int* __restrict__ ch_ptr,
                                                   const int* __restrict__ ch_idx, const int* __restrict__ ch_quad,
                                                   const int* __restrict__ lo_row, int PM,
                                                   const int* __restrict__ pjp, const float* __restrict__ pw,
                                                   const float* __restrict__ wthp, const float4* __restrict__ sh4,
                                                   const float2* __restrict__ inP, int TM,
                                                   const int* __restrict__ ttp, const float* __restrict__ tw,
                                                   float2* __restrict__ inC) {
  typedef Part<float> P;
  typedef P::H H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Gt = reinterpret_cast<float2*>(smem_raw);   // [4 quadrants][GR][2 JC][4]
  int blk = blockIdx.x;
  const int jcb = blk % njc;
  blk /= njc;
  const int it = blk % nit, B = blk / nit;
  const int i0 = it * TI, ni = min(TI, nthC - i0);
  const int half = nphC >> 1;
  const int j0 = jcb * JC, nj = min(JC, half - j0);
  const int lo = lo_row[it], hi = lo_row[nit + it];
  const int nr = hi - lo, W = 2 * nj;
  const int Kp = nthP * nphP, Kc = nthC * nphC;
  const float2* srcP = inP + (size_t)B * Kp * 4;
  const int NTH = blockDim.x / 2, task0 = threadIdx.x / 2, h = threadIdx.x % 2;
  const int r0 = task0 / W, u0 = task0 - r0 * W;
  const int dq = NTH / W, dr = NTH - dq * W;
  const size_t qstride = (size_t)nr * W;               // tasks per quadrant
  for (int r = r0, u = u0, task = task0; r < nr; task += NTH) {
    const int j = (u < nj) ? j0 + u : j0 + half + (u - nj);
    const int tp = lo + r;
    const float wt = wthp[tp];
    const float2* prow = srcP + (size_t)tp * nphP * 4;
    const float4* srow = sh4 + (size_t)tp * nphP * 2;
    H a0 = P::zero(), a1 = P::zero(), a2 = P::zero(), a3 = P::zero();
    const int pm = PMC > 0 ? 8 : PM;
#pragma unroll
    for (int q = 0; q < (PMC > 0 ? PMC : PM); q += 4) {
      const int4 jj = *reinterpret_cast<const int4*>(pjp + (size_t)j * pm + q);
      float w[4];
      P::w4(pw + (size_t)j * pm + q, w);
      const int js[4] = {jj.x, jj.y, jj.z, jj.w};
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (PMC > 0 && q + b >= PMC) break;
        const H v = ldp<float>(prow, js[b], h);
        const float4 s01 = srow[2 * js[b]], s23 = srow[2 * js[b] + 1];
        const float ww = w[b] * wt;
        P::cfma(a0, make_float2(ww * s01.x, -ww * s01.y), v);
        P::cfma(a1, make_float2(ww * s01.z, -ww * s01.w), v);
        P::cfma(a2, make_float2(ww * s23.x, -ww * s23.y), v);
        P::cfma(a3, make_float2(ww * s23.z, -ww * s23.w), v);
      }
    }
    stp<float>(Gt, task, h, a0);
    stp<float>(Gt, qstride + task, h, a1);
    stp<float>(Gt, 2 * qstride + task, h, a2);
    stp<float>(Gt, 3 * qstride + task, h, a3);
    u += dr;
    r += dq;
    if (u >= W) { u -= W; ++r; }
  }
  __syncthreads();
  const int c0 = ch_ptr[B], nch = ch_ptr[B + 1] - c0;
  for (int k = 0; k < nch; ++k) {
    const int cb = ch_idx[c0 + k];
    const float2* Gq = Gt + (size_t)ch_quad[c0 + k] * qstride * 4;
    for (int il = r0, u = u0; il < ni;) {
      const int ur = u < nj ? u + nj : u - nj;           // column j + N/2 (mod N)
      const int j = (u < nj) ? j0 + u : j0 + half + (u - nj);
      const int i = i0 + il;
      H a = P::zero();
      const int tm = PMC > 0 ? 8 : TM;
#pragma unroll
      for (int q = 0; q < (PMC > 0 ? PMC : TM); q += 4) {
        const int4 pk = *reinterpret_cast<const int4*>(ttp + (size_t)i * tm + q);
        float w[4];
        P::w4(tw + (size_t)i * tm + q, w);
        const int ps[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (PMC > 0 && q + b >= PMC) break;
          const int rr = (ps[b] & 0xffff) - lo;
          const size_t g = (size_t)rr * W + ((ps[b] >> 16) ? ur : u);
          P::rfma(a, w[b], ldp<float>(Gq, g, h));
        }
      }
      const size_t d = (size_t)cb * Kc + (size_t)i * nphC + j;
      H cur = ldp<float>(inC, d, h);
      P::add(cur, a);
      stp<float>(inC, d, h, cur);
      u += dr;
      il += dq;
      if (u >= W) { u -= W; ++il; }
    }
  }
}

// ------------------------------------------------------------------ receive
// y_e[m] += -jk sum_k w conj(sh) [P_th (z B0 + B3) + P_ph (z B1 - B2)]
// y_m[m] += -jk sum_k w conj(sh) [P_th (-B1 + B2/z) + P_ph (B0 + B3/z)]   (Eqs. 24-25)
// One CTA = a tile of up to 16 (particle, r) columns of one shape; threads are
// (mode, column pair); pattern and combined spectra chunks staged in shared memory.
template <typename T>
__global__ void k_receive(int K0, int npsi, int R, int RC, const int* __restrict__ tile_shape,
                          const int* __restrict__ tile_start, const int* __restrict__ tile_count,
                          const int* __restrict__ perm, const typename CV<T>::V* __restrict__ in0,
                          const typename CV<T>::V* __restrict__ P, const double* __restrict__ w0,
                          const double* __restrict__ dshift, int any_dshift,
                          const double* __restrict__ khat, double k, double zeta,
                          double2* __restrict__ y, int accumulate) {
  typedef typename CV<T>::V V;
  const int KC = 32;
  extern __shared__ unsigned char smem_raw[];
  V* Ps = reinterpret_cast<V*>(smem_raw);          // [KC][2][npsi]
  V* Cs = Ps + KC * 2 * npsi;                      // [KC][16 cols][4]
  int nrc = (R + RC - 1) / RC;
  int TP = max(1, 16 / RC);
  int nsub = (16 + TP - 1) / TP;
  int tile = blockIdx.x / (nsub * nrc);
  int sub = (blockIdx.x / nrc) % nsub, r0 = (blockIdx.x % nrc) * RC;
  int nr = min(RC, R - r0);
  int s = tile_shape[tile], tp = tile_count[tile];
  int t0 = tile_start[tile] + sub * TP;
  int ncol = max(0, min(tp - sub * TP, TP)) * nr;
  if (ncol == 0) return;                           // uniform per block: no barrier skipped
  int m = threadIdx.x % npsi, g = threadIdx.x / npsi;   // g in [0, 8): columns g, g + 8
  T z = (T)zeta, iz = (T)(1.0 / zeta);
  V ye[2] = {czero<V>(), czero<V>()}, ym[2] = {czero<V>(), czero<V>()};
  const V* Pg = P + (size_t)s * npsi * 2 * K0;
  for (int k0 = 0; k0 < K0; k0 += KC) {
    int nk = min(KC, K0 - k0);
    __syncthreads();
    for (int t = threadIdx.x; t < nk * 2 * npsi; t += blockDim.x) {
      int kl = t % nk, comp = (t / nk) % 2, mm = t / (2 * nk);
      Ps[(kl * 2 + comp) * npsi + mm] = Pg[((size_t)mm * 2 + comp) * K0 + k0 + kl];
    }
    for (int t = threadIdx.x; t < nk * ncol; t += blockDim.x) {
      int kl = t % nk, col = t / nk;
      int mu = perm[t0 + col / nr], r = r0 + col % nr;
      int kk = k0 + kl;
      const V* b = in0 + ((size_t)mu * K0 + kk) * 4 * R + r;
      V B0 = b[0], B1 = b[R], B2 = b[2 * R], B3 = b[3 * R];
      T wk = (T)w0[kk];
      V sh = mkc(wk, (T)0);
      if (any_dshift) {
        const double* d = dshift + 3 * mu;
        const double* kh = khat + 3 * kk;
        double ph = -k * (kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2]);
        double sn, cs;
        sincos(ph, &sn, &cs);
        sh = mkc((T)(w0[kk] * cs), (T)(w0[kk] * sn));
      }
      V* cc = Cs + ((size_t)kl * 16 + col) * 4;
      cc[0] = cmul(sh, mkc(z * B0.x + B3.x, z * B0.y + B3.y));
      cc[1] = cmul(sh, mkc(z * B1.x - B2.x, z * B1.y - B2.y));
      cc[2] = cmul(sh, mkc(-B1.x + iz * B2.x, -B1.y + iz * B2.y));
      cc[3] = cmul(sh, mkc(B0.x + iz * B3.x, B0.y + iz * B3.y));
    }
    __syncthreads();
    if (g < 8) {
      for (int kl = 0; kl < nk; ++kl) {
        V pt = Ps[(kl * 2) * npsi + m], pp = Ps[(kl * 2 + 1) * npsi + m];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          int col = g + 8 * q;
          if (col < ncol) {
            const V* cc = Cs + ((size_t)kl * 16 + col) * 4;
            cfma(ye[q], pt, cc[0]);
            cfma(ye[q], pp, cc[1]);
            cfma(ym[q], pt, cc[2]);
            cfma(ym[q], pp, cc[3]);
          }
        }
      }
    }
  }
  if (g >= 8) return;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int col = g + 8 * q;
    if (col >= ncol) continue;
    int mu = perm[t0 + col / nr], r = r0 + col % nr;
    double2 oe = make_double2(k * (double)ye[q].y, -k * (double)ye[q].x);   // -j k
    double2 om = make_double2(k * (double)ym[q].y, -k * (double)ym[q].x);
    double2* pe = y + ((size_t)mu * 2 * npsi + m) * R + r;
    double2* pm = pe + (size_t)npsi * R;
    if (accumulate) {
      double2 a = *pe, b = *pm;
      oe.x += a.x; oe.y += a.y; om.x += b.x; om.y += b.y;
    }
    *pe = oe;
    *pm = om;
  }
}

// ------------------------------------------------------------------ block-sparse product
// y[mu][i][r] (+)= sum_{e in row mu} sum_j B[blk_e][i][j] x[col_e][j][r]
template <typename T, typename XV = double2>
__global__ void k_blocksparse(int nrow, int n2, int R, int rc, int nrc, const int* __restrict__ ptr,
                              const int* __restrict__ col, const int* __restrict__ blk,
                              const typename CV<T>::V* __restrict__ Bt,
                              const XV* __restrict__ x, double2* __restrict__ y,
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
    const XV* xv = x + (size_t)col[e] * n2 * R + r0;
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
int ensure_spectra(Ctx* c, int R, int prec) {
  int p = (prec == SMR_PREC_FP64) ? 0 : 1;
  if (c->buf_R[p] != R) {
    // (re)allocate this precision's spectra; graphs built on them are dropped
    for (size_t i = 0; i < c->graphs.size();) {
      if (c->graphs[i].prec == prec) {
        cudaGraphExecDestroy(c->graphs[i].exec);
        c->graphs.erase(c->graphs.begin() + i);
      } else {
        ++i;
      }
    }
    size_t es = (p == 0) ? sizeof(double2) : sizeof(float2);
    size_t gmax = 0;
    c->buf_R[p] = 0;
    for (int s = 0; s < c->nlev; ++s) {
      Level& L = c->lev[s];
      if (L.buf_out[p]) cudaFree(L.buf_out[p]);
      if (L.buf_in[p]) cudaFree(L.buf_in[p]);
      L.buf_out[p] = L.buf_in[p] = nullptr;
      size_t bytes = (size_t)L.nbox * L.K * 4 * R * es;
      if (cudaMalloc(&L.buf_out[p], bytes) != cudaSuccess || cudaMalloc(&L.buf_in[p], bytes) != cudaSuccess) {
        c->err = "out of device memory for level spectra";
        c->spec_prec = -1;
        return SMR_E_OOM;
      }
      L.buf_bytes[p] = bytes;
      if (s + 1 < c->nlev)
        gmax = std::max(gmax, (size_t)L.nbox * c->lev[s + 1].nth * L.nph * 4 * R * es);
    }
    if (c->pspec[p]) cudaFree(c->pspec[p]);
    c->pspec[p] = nullptr;
    if ((c->multi || c->any_dshift) &&
        cudaMalloc(&c->pspec[p], (size_t)c->p * c->lev[0].K * 4 * R * es) != cudaSuccess) {
      c->err = "out of device memory for the per-particle spectra";
      c->spec_prec = -1;
      return SMR_E_OOM;
    }
    if (c->G_buf[p]) cudaFree(c->G_buf[p]);
    c->G_buf[p] = nullptr;
    if (gmax && cudaMalloc(&c->G_buf[p], gmax) != cudaSuccess) {
      c->err = "out of device memory for the separable-pass buffer";
      c->spec_prec = -1;
      return SMR_E_OOM;
    }
    c->G_size[p] = gmax;
    c->buf_R[p] = R;
  }
  for (auto& L : c->lev) {
    L.d_out = L.buf_out[p];
    L.d_in = L.buf_in[p];
    L.spec_bytes = L.buf_bytes[p];
  }
  c->d_G = c->G_buf[p];
  c->G_bytes = c->G_size[p];
  c->spec_R = R;
  c->spec_prec = prec;
  return SMR_OK;
}

// Direction chunk of the whole-level translation: the largest power of two
// up to 32 whose staged spectra and tables fit in 96 KB (0: none fits).
int translate_lvl_chunk(int nbox, size_t vbytes) {
  for (int kch = 32; kch >= 4; kch /= 2)
    if (((size_t)nbox * kch * 4 + (size_t)49 * kch) * vbytes <= 96 * 1024) return kch;
  return 0;
}

bool translate_lvl_ok(Ctx* c, int s, bool f64) {
  const Level& L = c->lev[s];
  if (L.off_dx.empty() || !L.d_il_pk || translate_lvl_chunk(L.nbox, f64 ? 16 : 8) == 0) return false;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_translate_lvl<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_translate_lvl<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  return true;
}

// The per-parent FP32 anterpolation needs the 8-tap tables and its four
// quadrants' phi-pass rows within the fixed shared-memory ceiling.
bool anterp4_ok(Ctx* c, int s) {
  const Level& Lc = c->lev[s];
  if (!Lc.d_shift4_32 || Lc.ant_PM != 8 || Lc.ant_TM != 8 || std::max(Lc.ant_PMx, Lc.ant_TMx) > 8) return false;
  const size_t sm4 = (size_t)4 * Lc.ant_GR * 2 * Lc.ant_JC5 * 4 * sizeof(float2);
  if (Lc.ant_JC5 < 1 || sm4 > 200 * 1024) return false;
  static bool attr = false;
  if (!attr) {
    // one fixed ceiling for every launch (graph nodes keep their own size)
    cudaFuncSetAttribute(k_anterp4<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_anterp4<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  return true;
}

// Finest boxes made of cells.  Box b's outgoing spectrum is the sum of its
// particles' spectra, and each particle receives its box's incoming
// spectrum; a row is one box's or one particle's [K0][4][R] spectrum.  With
// `shift` set the kernels also carry each particle's displacement d from
// its box centre: e^{+jk khat.d} into the sum, e^{-jk khat.d} out of the
// broadcast (the tensor-core aggregation and receive work on unshifted
// per-particle spectra).  Grid: (boxes or particles, row chunks of 256
// elements); both kernels guard the row end.
template <typename T>
__device__ __forceinline__ typename CV<T>::V shift_phase(const double* d, const double* kh, double k, double sgn) {
  const double ph = sgn * k * (kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2]);
  T sn, cs;
  if (sizeof(T) == 8) {
    double s8, c8;
    sincos(ph, &s8, &c8);
    sn = (T)s8;
    cs = (T)c8;
  } else {
    float s4, c4;
    sincosf((float)ph, &s4, &c4);
    sn = (T)s4;
    cs = (T)c4;
  }
  return mkc(cs, sn);
}

template <typename T>
__global__ void k_cell_sum(int nbox, long long row, int R, const int* __restrict__ ptr,
                           const int* __restrict__ idx, int shift, const double* __restrict__ dshift,
                           const double* __restrict__ khat, double k,
                           const typename CV<T>::V* __restrict__ part, typename CV<T>::V* __restrict__ box) {
  typedef typename CV<T>::V V;
  const int b = blockIdx.x;
  const long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x;
  if (b >= nbox || e >= row) return;
  const int kk = (int)(e / (4LL * R));
  V acc = mkc((T)0, (T)0);
  for (int t = ptr[b]; t < ptr[b + 1]; ++t) {
    const int mu = idx[t];
    V v = part[(size_t)mu * row + e];
    if (shift) v = cmul(v, shift_phase<T>(dshift + 3 * mu, khat + 3 * kk, k, 1.0));
    acc.x += v.x;
    acc.y += v.y;
  }
  box[(size_t)b * row + e] = acc;
}

template <typename T>
__global__ void k_cell_bcast(int p, long long row, int R, const int* __restrict__ cell, int shift,
                             const double* __restrict__ dshift, const double* __restrict__ khat, double k,
                             const typename CV<T>::V* __restrict__ box, typename CV<T>::V* __restrict__ part) {
  typedef typename CV<T>::V V;
  const int mu = blockIdx.x;
  const long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x;
  if (mu >= p || e >= row) return;
  V v = box[(size_t)cell[mu] * row + e];
  if (shift) v = cmul(v, shift_phase<T>(dshift + 3 * mu, khat + 3 * (int)(e / (4LL * R)), k, -1.0));
  part[(size_t)mu * row + e] = v;
}

template <typename T>
static int far_impl(Ctx* c, int R, const double2* x, double2* y, bool accumulate, cudaStream_t st) {
  typedef typename CV<T>::V V;
  const bool f64 = sizeof(T) == 8;
  const double es = sizeof(V), R_ = R;
  Level& L0 = c->lev[0];
  int RC = std::min(R, 16);
  int nrc = (R + RC - 1) / RC;
  // Overlap: the translation of each level runs on a side stream after an
  // event that marks its outgoing spectra, and the anterpolation into a level
  // waits for that level's translation; the receive waits for the near
  // product when run_product put it on a side stream (c->near_ev).
  Ctx::Side* sd = (c->overlap && !c->prof && c->cur_side < (int)c->side.size()) ? &c->side[c->cur_side] : nullptr;
  if (sd && (!sd->tr || c->nlev > (int)sd->eout.size())) sd = nullptr;
  // translation at every level (in the upward loop when it overlaps)
  auto translate = [&](int s, cudaStream_t ts) -> int {
    Level& L = c->lev[s];
    if (L.off_dx.empty()) {                  // no interaction list at this level
      SMR_CUDA(c, cudaMemsetAsync(L.d_in, 0, L.spec_bytes, ts));
      return SMR_OK;
    }
    int noff = 49;                           // tables by lattice offset (7 x 7 grid)
    int cap = f64 ? 16 : 32;                 // directions x columns staged per CTA
    int RCt = std::min(R, cap);
    int KC = std::max(1, cap / RCt);
    int nkch = (L.K + KC - 1) / KC;
    int nrct = (R + RCt - 1) / RCt;
    size_t sm = ((size_t)64 * KC * 4 * RCt + (size_t)std::max(noff, 1) * KC) * sizeof(V) +
                (64 + 16 + 16) * sizeof(int) + 16 * 27 * sizeof(int2);
    cudaFuncSetAttribute(k_translate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    pbeg(c, ts, "translate", s,
         2.0 * L.nbox * L.K * 4 * R_ * es + (double)L.off_dx.size() * L.K * es,
         8.0 * L.il_src.size() * L.K * 4 * R_);
    // single right-hand side: 8x8-tile register-blocked kernel, except on
    // levels whose few boxes would leave most of one 8x8 tile idle (or as tuned)
    const int tv = (R == 1) ? L.tune_tr[f64 ? 0 : 1] : 0;
    if (tv == 5 && translate_lvl_ok(c, s, f64)) {
      const int KCH = translate_lvl_chunk(L.nbox, sizeof(V));
      const size_t sml = ((size_t)L.nbox * KCH * 4 + (size_t)49 * KCH) * sizeof(V);
      k_translate_lvl<T><<<(unsigned)((L.K + KCH - 1) / KCH), 256, sml, ts>>>(
          L.K, L.nbox, KCH, L.d_il_ptr, L.d_il_pk, (const V*)(f64 ? (void*)L.d_T64 : (void*)L.d_T32),
          (const V*)L.d_out, (V*)L.d_in);
      SMR_LAUNCH(c);
      pend(c, ts);
      return SMR_OK;
    }
    const bool few = (tv == 4) || (tv == 0 && R == 1 && L.nbox <= 64);
    const bool use8 = (tv == 0) ? (R == 1 && !(L.ntile8_ne == 1 && L.nbox < 32)) : (tv != 3);
    if (few) {
      const int TG = 8;
      dim3 g((unsigned)(((long long)L.K * Part<T>::NT + 255) / 256), (unsigned)((L.nbox + TG - 1) / TG));
      k_translate_few<T><<<g, 256, 0, ts>>>(L.K, L.nbox, TG, L.d_il_ptr, L.d_il_pk,
                                             (const V*)(f64 ? (void*)L.d_T64 : (void*)L.d_T32), (const V*)L.d_out,
                                             (V*)L.d_in);
    } else if (use8) {
      // direction chunk: 16 (FP32) or 8 (FP64) directions, halved by the tuner
      const bool halfc = (tv == 2);
      int KC1 = (f64 ? 8 : 16) / (halfc ? 2 : 1);
      int nk1 = (L.K + KC1 - 1) / KC1;
      // FP32 tables are staged as 16-byte (t_r, t_r, -t_i, t_i) entries
      size_t sm1 = ((size_t)144 * KC1 * 4) * sizeof(V) + (size_t)49 * KC1 * (f64 ? sizeof(V) : 16) +
                   (144 + 64) * sizeof(int);
      auto kt = halfc ? k_translate1<T, (sizeof(T) == 8 ? 4 : 8)> : k_translate1<T, (sizeof(T) == 8 ? 8 : 16)>;
      cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      kt<<<(unsigned)(L.ntile8_ne * nk1), 16 * KC1 * Part<T>::NT, sm1, ts>>>(
          L.K, L.ntile8_x, L.ntile8_ne, L.d_tiles8, L.map_x0, L.map_y0, L.map_w, L.map_h, L.d_boxmap,
          (const V*)(f64 ? (void*)L.d_T64 : (void*)L.d_T32), (const V*)L.d_out, (V*)L.d_in);
    } else {
      k_translate<T><<<(unsigned)(L.ntile_ne * nkch * nrct), 256, sm, ts>>>(
          L.K, R, RCt, KC, L.ntile_x, L.ntile_ne, L.d_tiles, L.map_x0, L.map_y0, L.map_w, L.map_h, noff,
          L.d_boxmap, L.d_offid,
          (const V*)(f64 ? (void*)L.d_T64 : (void*)L.d_T32), (const V*)L.d_out, (V*)L.d_in);
    }
    SMR_LAUNCH(c);
    pend(c, ts);
    return SMR_OK;
  };
  auto fork_translate = [&](int s) -> int {
    SMR_CUDA(c, cudaEventRecord(sd->eout[s], st));
    SMR_CUDA(c, cudaStreamWaitEvent(sd->tr, sd->eout[s], 0));
    int rc = translate(s, sd->tr);
    if (rc) return rc;
    SMR_CUDA(c, cudaEventRecord(sd->etr[s], sd->tr));
    return SMR_OK;
  };
  // aggregation
  {
    int nkc = (L0.K + 63) / 64;
    size_t sm = (size_t)16 * 2 * c->npsi * sizeof(V);
    pbeg(c, st, "aggregate", 0,
         (double)c->p * 2 * c->npsi * R_ * 16 + (double)c->S * c->npsi * 2 * L0.K * es +
             (double)c->p * L0.K * 4 * R_ * es,
         32.0 * c->npsi * c->p * L0.K * R_);
    // per-particle spectra go through the box sum where boxes hold several
    // particles, or where the tensor cores aggregate displaced particles
    // (the sum then applies the displacement shifts)
    const bool tc = !f64 && tc_aggregate_ok(c, R) && c->tune_tc_agg != 0;
    const bool cells = c->multi || (tc && c->any_dshift);
    V* agg = (V*)(cells ? c->pspec[f64 ? 0 : 1] : L0.d_out);
    if (tc) {
      int rc = run_aggregate_tc(c, x, c->x32_of == x ? c->d_x32 : nullptr, (float2*)agg, st);
      if (rc) {
        pend(c, st);
        return rc;
      }
    } else {
      int nsub = (16 + std::max(1, 16 / RC) - 1) / std::max(1, 16 / RC);
      k_aggregate<T><<<(unsigned)(c->ntile * nsub * nkc * nrc), 256, sm, st>>>(
          L0.K, c->npsi, R, RC, nkc, c->d_tile_shape, c->d_tile_start, c->d_tile_count, c->d_perm, x,
          (const V*)(f64 ? (void*)c->d_P64 : (void*)c->d_P32), c->d_dshift, c->any_dshift, L0.d_khat,
          c->k, agg);
      SMR_LAUNCH(c);
    }
    if (cells) {
      const long long row = (long long)L0.K * 4 * R;
      k_cell_sum<T><<<dim3((unsigned)L0.nbox, (unsigned)((row + 255) / 256)), 256, 0, st>>>(
          L0.nbox, row, R, c->d_cell_ptr, c->d_cell_idx, (tc && c->any_dshift) ? 1 : 0, c->d_dshift,
          L0.d_khat, c->k, agg, (V*)L0.d_out);
      SMR_LAUNCH(c);
    }
    pend(c, st);
  }
  // upward: separable interpolation, theta then phi (+ shift + child sum)
  for (int s = 0; s + 1 < c->nlev; ++s) {
    if (sd) {
      int rc = fork_translate(s);              // level s's outgoing spectra are complete
      if (rc) return rc;
    }
    Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
    pbeg(c, st, "interpolate", s,
         ((double)Lc.nbox * Lc.K + (double)Lp.nbox * Lp.K) * 4 * R_ * es + 4.0 * Lp.K * es,
         (double)Lc.nbox * Lp.nth * Lc.nph * 4 * R_ * 16.0 + (double)Lc.nbox * Lp.K * 4 * R_ * 24.0);
    if (!f64 && R == 1 && (Lc.tune_ip[1] == 0 || Lc.tune_ip[1] == 3) && interp2_ok(c, s)) {
      int rc = run_interp2(c, s, st);
      pend(c, st);
      if (rc) return rc;
      continue;
    }
    if (R == 1 && Lp.nph * Part<T>::NT <= 256 * EM1<T>::v) {
      int TR = std::max(1, std::min(Lp.nth, (256 * EM1<T>::v) / (Lp.nph * Part<T>::NT)));
      if (Lc.tune_ip[f64 ? 0 : 1] == 2) TR = std::max(1, TR / 2);
      int nrt = (Lp.nth + TR - 1) / TR;
      size_t sm1 = (size_t)TR * Lc.nph * 4 * sizeof(V);
      cudaFuncSetAttribute(k_interp1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
      const unsigned mP = (unsigned)(((1ull << 32) + (unsigned)Lp.nph - 1) / (unsigned)Lp.nph);
      k_interp1<T><<<(unsigned)(Lp.nbox * nrt), 256, sm1, st>>>(
          Lp.nth, Lp.nph, mP, Lc.nph, Lc.K, TR, nrt, Lp.d_ch_ptr, Lp.d_ch_idx, Lp.d_ch_quad, Lc.d_th_pk,
          (const T*)(f64 ? (void*)Lc.d_th_ws64 : (void*)Lc.d_th_ws32), Lc.d_ph_src,
          (const T*)(f64 ? (void*)Lc.d_ph_w64 : (void*)Lc.d_ph_w32),
          (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)Lc.d_out, (V*)Lp.d_out);
      SMR_LAUNCH(c);
      pend(c, st);
      continue;
    }
    // fused (shared-memory) version when a tile of parent rows fits
    int TR = std::max(1, std::min(Lp.nth, (256 * EMAX) / (Lp.nph * 4 * R)));
    size_t smf = (size_t)TR * Lc.nph * 4 * R * sizeof(V);
    if (Lp.nph * 4 * R <= 256 * EMAX && smf <= 96 * 1024) {
      int nrt = (Lp.nth + TR - 1) / TR;
      auto kf = (R == 1) ? k_interp_fused<T, true> : k_interp_fused<T, false>;
      cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
      kf<<<(unsigned)(Lp.nbox * nrt), 256, smf, st>>>(
          Lp.nth, Lp.nph, Lc.nph, Lc.K, R, TR, nrt, Lp.d_ch_ptr, Lp.d_ch_idx, Lp.d_ch_quad, Lc.d_th_src,
          Lc.d_th_refl, (const T*)(f64 ? (void*)Lc.d_th_w64 : (void*)Lc.d_th_w32), Lc.d_ph_src,
          (const T*)(f64 ? (void*)Lc.d_ph_w64 : (void*)Lc.d_ph_w32),
          (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)Lc.d_out, (V*)Lp.d_out);
      SMR_LAUNCH(c);
      pend(c, st);
      continue;
    }
    int rows1 = Lc.nbox * Lp.nth;
    auto kth = (R == 1) ? k_interp_theta<T, true> : k_interp_theta<T, false>;
    kth<<<(unsigned)((rows1 + 7) / 8), 256, 0, st>>>(
        rows1, Lp.nth, Lc.nph, Lc.K, R, Lc.d_th_src, Lc.d_th_refl,
        (const T*)(f64 ? (void*)Lc.d_th_w64 : (void*)Lc.d_th_w32), (const V*)Lc.d_out, (V*)c->d_G);
    SMR_LAUNCH(c);
    int rows2 = Lp.nbox * Lp.nth;
    auto kph = (R == 1) ? k_interp_phi<T, true> : k_interp_phi<T, false>;
    kph<<<(unsigned)((rows2 + 7) / 8), 256, 0, st>>>(
        rows2, Lp.nth, Lp.nph, Lc.nph, R, Lp.d_ch_ptr, Lp.d_ch_idx, Lp.d_ch_quad, Lc.d_ph_src,
        (const T*)(f64 ? (void*)Lc.d_ph_w64 : (void*)Lc.d_ph_w32),
        (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)c->d_G, (V*)Lp.d_out);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  if (sd) {
    int rc = fork_translate(c->nlev - 1);      // the top level
    if (rc) return rc;
  } else {
    for (int s = 0; s < c->nlev; ++s) {
      int rc = translate(s, st);
      if (rc) return rc;
    }
  }
  // downward: separable adjoint, phi-transpose then theta-transpose (accumulates)
  for (int s = c->nlev - 2; s >= 0; --s) {
    if (sd) {
      // the parent level's incoming spectra and this level's translation
      SMR_CUDA(c, cudaStreamWaitEvent(st, sd->etr[s + 1], 0));
      SMR_CUDA(c, cudaStreamWaitEvent(st, sd->etr[s], 0));
    }
    Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
    pbeg(c, st, "anterpolate", s,
         ((double)Lp.nbox * Lp.K + 2.0 * Lc.nbox * Lc.K) * 4 * R_ * es + 4.0 * Lp.K * es,
         (double)Lc.nbox * Lp.nth * Lc.nph * 4 * R_ * 8.0 * 2 * (double)Lp.nph / Lc.nph * 4.0 / 4.0 +
             (double)Lc.nbox * Lc.K * 4 * R_ * 16.0 * (double)Lp.nth / Lc.nth);
    if (!f64 && R == 1 && Lc.tune_an[1] == 4 && anterp2_ok(c, s)) {
      int rc = run_anterp2(c, s, st);
      pend(c, st);
      if (rc) return rc;
      continue;
    }
    if (!f64 && R == 1 && Lc.tune_an[1] == 5 && anterp4_ok(c, s)) {
      const int JC = Lc.ant_JC5;
      const int njc = (Lc.nph / 2 + JC - 1) / JC;
      const size_t sm4 = (size_t)4 * Lc.ant_GR * 2 * JC * 4 * sizeof(float2);
      auto ka = std::max(Lc.ant_PMx, Lc.ant_TMx) <= 7 ? k_anterp4<7> : k_anterp4<8>;
      ka<<<(unsigned)(Lp.nbox * Lc.ant_nit * njc), 256, sm4, st>>>(
          Lc.nth, Lc.nph, Lp.nth, Lp.nph, Lc.ant_TI, Lc.ant_nit, JC, njc, Lp.d_ch_ptr, Lp.d_ch_idx, Lp.d_ch_quad,
          Lc.d_ant_lo, Lc.ant_PM, Lc.d_ant_pjp, Lc.d_ant_pw32, Lc.d_wthp32, (const float4*)Lc.d_shift4_32,
          (const float2*)Lp.d_in, Lc.ant_TM, Lc.d_ant_ttp, Lc.d_ant_tw32, (float2*)Lc.d_in);
      SMR_LAUNCH(c);
      pend(c, st);
      continue;
    }
    if (R == 1) {
      const int an = Lc.tune_an[f64 ? 0 : 1];
      int JC = Lc.ant_JC[f64 ? 0 : 1];
      if (an == 1) JC = std::max(1, JC / 2);
      int njc = (Lc.nph / 2 + JC - 1) / JC;
      size_t sm1 = (size_t)Lc.ant_GR * 2 * JC * 4 * sizeof(V);
      int thr = (an == 2 || Lc.ant_GR * 2 * JC * (Part<T>::NT / (f64 ? 2 : 1)) >= 2048) ? 256 : 128;
      auto ka = k_anterp1<T, 0>;
      if (Lc.ant_PM == 8 && Lc.ant_TM == 8) ka = std::max(Lc.ant_PMx, Lc.ant_TMx) <= 7 ? k_anterp1<T, 7> : k_anterp1<T, 8>;
      ka<<<(unsigned)(Lc.nbox * Lc.ant_nit * njc), thr, sm1, st>>>(
          Lc.nth, Lc.nph, Lp.nth, Lp.nph, Lc.ant_TI, Lc.ant_nit, JC, njc, Lc.d_parent, Lc.d_quad, Lc.d_ant_lo,
          Lc.ant_PM, Lc.d_ant_pjp, (const T*)(f64 ? (void*)Lc.d_ant_pw64 : (void*)Lc.d_ant_pw32),
          (const T*)(f64 ? (void*)Lc.d_wthp64 : (void*)Lc.d_wthp32),
          (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)Lp.d_in, Lc.ant_TM,
          Lc.d_ant_ttp, (const T*)(f64 ? (void*)Lc.d_ant_tw64 : (void*)Lc.d_ant_tw32), (V*)Lc.d_in);
      SMR_LAUNCH(c);
      pend(c, st);
      continue;
    }
    int rows1 = Lc.nbox * Lp.nth;
    auto kap = (R == 1) ? k_anterp_phi<T, true> : k_anterp_phi<T, false>;
    kap<<<(unsigned)((rows1 + 7) / 8), 256, 0, st>>>(
        rows1, Lp.nth, Lp.nph, Lc.nph, R, Lc.d_parent, Lc.d_quad, Lc.d_pht_ptr, Lc.d_pht_jp,
        (const T*)(f64 ? (void*)Lc.d_pht_w64 : (void*)Lc.d_pht_w32),
        (const T*)(f64 ? (void*)Lc.d_wthp64 : (void*)Lc.d_wthp32),
        (const V*)(f64 ? (void*)Lc.d_shift64 : (void*)Lc.d_shift32), (const V*)Lp.d_in, (V*)c->d_G);
    SMR_LAUNCH(c);
    int rows2 = Lc.nbox * Lc.nth;
    auto kat = (R == 1) ? k_anterp_theta<T, true> : k_anterp_theta<T, false>;
    kat<<<(unsigned)((rows2 + 7) / 8), 256, 0, st>>>(
        rows2, Lc.nth, Lp.nth, Lc.nph, R, Lc.d_tht_ptr, Lc.d_tht_tp, Lc.d_tht_refl,
        (const T*)(f64 ? (void*)Lc.d_tht_w64 : (void*)Lc.d_tht_w32), (const V*)c->d_G, (V*)Lc.d_in);
    SMR_LAUNCH(c);
    pend(c, st);
  }
  // receive
  if (sd) SMR_CUDA(c, cudaStreamWaitEvent(st, sd->etr[0], 0));
  if (c->near_ev) SMR_CUDA(c, cudaStreamWaitEvent(st, c->near_ev, 0));
  {
    int thr = c->npsi * 8;
    size_t sm = ((size_t)32 * 2 * c->npsi + 32 * 16 * 4) * sizeof(V);
    pbeg(c, st, "receive", 0,
         (double)c->p * L0.K * 4 * R_ * es + (double)c->S * c->npsi * 2 * L0.K * es +
             (accumulate ? 2.0 : 1.0) * c->p * 2 * c->npsi * R_ * 16,
         48.0 * c->p * c->npsi * L0.K * R_);
    // per-particle incoming spectra where boxes hold several particles, or
    // where the tensor cores receive for displaced particles (the broadcast
    // then applies the displacement shifts)
    const bool tc = !f64 && tc_receive_ok(c, R) && c->tune_tc_rec != 0;
    const bool cells = c->multi || (tc && c->any_dshift);
    const V* inc = (const V*)L0.d_in;
    if (cells) {
      const long long row = (long long)L0.K * 4 * R;
      V* part = (V*)c->pspec[f64 ? 0 : 1];
      k_cell_bcast<T><<<dim3((unsigned)c->p, (unsigned)((row + 255) / 256)), 256, 0, st>>>(
          c->p, row, R, c->d_cell_of, (tc && c->any_dshift) ? 1 : 0, c->d_dshift, L0.d_khat, c->k,
          (const V*)L0.d_in, part);
      SMR_LAUNCH(c);
      inc = part;
    }
    if (tc) {
      int rc = run_receive_tc(c, (const float2*)inc, y, accumulate, st);
      pend(c, st);
      return rc;
    }
    int nsub = (16 + std::max(1, 16 / RC) - 1) / std::max(1, 16 / RC);
    cudaFuncSetAttribute(k_receive<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k_receive<T><<<(unsigned)(c->ntile * nsub * nrc), thr, sm, st>>>(
        L0.K, c->npsi, R, RC, c->d_tile_shape, c->d_tile_start, c->d_tile_count, c->d_perm,
        inc, (const V*)(f64 ? (void*)c->d_P64 : (void*)c->d_P32), L0.d_w, c->d_dshift,
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

__global__ void k_x32f(long long n, const double2* __restrict__ a, float2* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// The FP32 single right-hand-side product converts x to FP32 once (the
// conversion runs on the FP64 units, 1/64 of the FP32 rate) for the near
// gathers and the tensor-core aggregation; c->x32_of records which x the
// copy holds, so a step that finds another x reads the FP64 one.  The record
// lives for one product call: the callers clear it before they return, and
// graph capture clears it (a capture converts nothing).
int prep_x32(Ctx* c, int R, int prec, const double2* x, cudaStream_t st) {
  c->x32_of = nullptr;
  if (prec != SMR_PREC_FP32 || R != 1 || !c->d_x32) return SMR_OK;
  const long long n = (long long)c->p * 2 * c->npsi;
  pbeg(c, st, "convert", -1, (double)n * 24.0, 0.0);
  k_x32f<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, c->d_x32);
  SMR_LAUNCH(c);
  pend(c, st);
  c->x32_of = x;
  return SMR_OK;
}

int run_near(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st) {
  if (prec == SMR_PREC_FP32 && tc_near_ok(c, R) && c->tune_tc_near != 0) {
    if (c->x32_of != x) {
      int rc = prep_x32(c, R, prec, x, st);
      if (rc) return rc;
    }
    return run_near_tc(c, y, st);
  }
  double n2 = 2.0 * c->npsi, es = prec == SMR_PREC_FP64 ? 16 : 8;
  const bool x32 = prec == SMR_PREC_FP32 && R == 1 && c->x32_of == x;
  pbeg(c, st, "near", -1, c->p * n2 * R * (x32 ? 8 + 16 : 16 + 16) + (double)c->nblk * n2 * n2 * es,
       8.0 * n2 * n2 * c->nr_col.size() * R);
  int rc;
  if (x32) {
    const int n2i = 2 * c->npsi;
    k_blocksparse<float, float2><<<(unsigned)c->p, n2i, (size_t)n2i * sizeof(float2), st>>>(
        c->p, n2i, 1, 1, 1, c->d_nr_ptr, c->d_nr_col, c->d_nr_blk, c->d_B32, c->d_x32, y, 0);
    SMR_LAUNCH(c);
    rc = SMR_OK;
  } else {
    rc = (prec == SMR_PREC_FP64)
             ? bs_impl<double>(c, c->p, R, c->d_nr_ptr, c->d_nr_col, c->d_nr_blk, c->d_B64, x, y, false, st)
             : bs_impl<float>(c, c->p, R, c->d_nr_ptr, c->d_nr_col, c->d_nr_blk, c->d_B32, x, y, false, st);
  }
  pend(c, st);
  return rc;
}

// out[c][i] = in[i][c] for in [rows][cols] (tiles of 32 x 32 through shared
// memory); grid x runs over the longer of the two dimensions
__global__ void k_transpose_c128(long long rows, long long cols, const double2* __restrict__ in,
                                 double2* __restrict__ out) {
  __shared__ double2 t[32][33];
  const bool rx = rows >= cols;
  const long long i0 = (long long)(rx ? blockIdx.x : blockIdx.y) * 32;
  const long long c0 = (long long)(rx ? blockIdx.y : blockIdx.x) * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    long long i = i0 + k, cc = c0 + threadIdx.x;
    if (i < rows && cc < cols) t[k][threadIdx.x] = in[i * cols + cc];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    long long cc = c0 + k, i = i0 + threadIdx.x;
    if (i < rows && cc < cols) out[cc * rows + i] = t[threadIdx.x][k];
  }
}

static int transpose_c128(Ctx* c, long long rows, long long cols, const double2* in, double2* out,
                          cudaStream_t st) {
  long long a = (rows + 31) / 32, b = (cols + 31) / 32;
  dim3 g((unsigned)std::max(a, b), (unsigned)std::min(a, b));
  k_transpose_c128<<<g, dim3(32, 8), 0, st>>>(rows, cols, in, out);
  SMR_LAUNCH(c);
  return SMR_OK;
}

bool split_columns(const Ctx* c, int R, int prec) { return R > 1 && prec == SMR_PREC_FP32 && c->split_cols; }

// column buffers [R][N] for split products (allocated outside graph capture)
int ensure_split(Ctx* c, int R) {
  size_t need = (size_t)2 * R * 2 * c->npsi * c->p;
  if (c->split_elems >= need) return SMR_OK;
  if (c->d_split) cudaFree(c->d_split);
  c->d_split = nullptr;
  c->split_elems = 0;
  if (cudaMalloc((void**)&c->d_split, need * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    c->err = "out of device memory for the column buffers of a split product";
    return SMR_E_OOM;
  }
  c->split_elems = need;
  return SMR_OK;
}

void free_lanes(Ctx* c) {
  for (size_t j = 1; j < c->lanes.size(); ++j) {
    Ctx::Lane& a = c->lanes[j];
    for (void* q : a.out) if (q) cudaFree(q);
    for (void* q : a.in) if (q) cudaFree(q);
    if (a.G) cudaFree(a.G);
    if (a.x32) cudaFree(a.x32);
    if (a.tcn_part) cudaFree(a.tcn_part);
    if (a.s) cudaStreamDestroy(a.s);
  }
  for (auto& a : c->lanes)
    if (a.ev) cudaEventDestroy(a.ev);
  c->lanes.clear();
  if (c->lane_fork) cudaEventDestroy(c->lane_fork);
  c->lane_fork = nullptr;
}

// Work buffers of nl column lanes for FP32 single-column products (outside
// graph capture; lanes that exist are kept and grown only).
int ensure_lanes(Ctx* c, int nl) {
  int rc = ensure_spectra(c, 1, SMR_PREC_FP32);
  if (rc) return rc;
  if ((int)c->lanes.size() < nl) c->lanes.resize(nl);
  if (!c->lane_fork) SMR_CUDA(c, cudaEventCreateWithFlags(&c->lane_fork, cudaEventDisableTiming));
  Ctx::Lane& l0 = c->lanes[0];                 // the context's own buffers
  l0.out.assign(c->nlev, nullptr);
  l0.in.assign(c->nlev, nullptr);
  for (int s = 0; s < c->nlev; ++s) {
    l0.out[s] = c->lev[s].buf_out[1];
    l0.in[s] = c->lev[s].buf_in[1];
  }
  l0.G = c->G_buf[1];
  l0.x32 = c->d_x32;
  l0.tcn_part = c->d_tcn_part;
  for (int j = 0; j < nl; ++j) {
    Ctx::Lane& a = c->lanes[j];
    if (!a.ev) SMR_CUDA(c, cudaEventCreateWithFlags(&a.ev, cudaEventDisableTiming));
    if (j == 0) continue;
    if (!a.s) SMR_CUDA(c, cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking));
    if ((int)a.out.size() != c->nlev) {
      a.out.assign(c->nlev, nullptr);
      a.in.assign(c->nlev, nullptr);
    }
    bool ok = true;
    for (int s = 0; s < c->nlev && ok; ++s) {
      const size_t b = c->lev[s].buf_bytes[1];
      ok = (a.out[s] || cudaMalloc(&a.out[s], b) == cudaSuccess) &&
           (a.in[s] || cudaMalloc(&a.in[s], b) == cudaSuccess);
    }
    if (ok && c->G_size[1] && !a.G) ok = cudaMalloc(&a.G, c->G_size[1]) == cudaSuccess;
    if (ok && c->d_x32 && !a.x32)
      ok = cudaMalloc((void**)&a.x32, (size_t)c->p * 2 * c->npsi * sizeof(float2)) == cudaSuccess;
    if (ok && c->d_tcn_part && !a.tcn_part) ok = cudaMalloc((void**)&a.tcn_part, c->tcn_part_bytes) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_lanes(c);
      c->err = "out of device memory for the column lanes of a split product";
      return SMR_E_OOM;
    }
  }
  return SMR_OK;
}

// Points the FP32 single-column work buffers at lane j's.
static void use_lane(Ctx* c, int j) {
  const Ctx::Lane& a = c->lanes[j];
  for (int s = 0; s < c->nlev; ++s) {
    c->lev[s].d_out = a.out[s];
    c->lev[s].d_in = a.in[s];
  }
  c->d_G = a.G;
  c->d_x32 = a.x32;
  c->d_tcn_part = a.tcn_part;
}

// one lane where products use the shared per-particle spectra (several
// particles per box, or displaced particles)
int lanes_for(const Ctx* c, int R) {
  return (c->prof || c->multi || c->any_dshift) ? 1 : std::max(1, std::min(R, c->n_lanes));
}

// Side streams and events of lanes 0 .. n-1 for the overlapped product
// (created outside graph capture, kept until the context goes).
int ensure_side(Ctx* c, int n) {
  if (!c->overlap) return SMR_OK;
  if ((int)c->side.size() < n) c->side.resize(n);
  for (int j = 0; j < n; ++j) {
    Ctx::Side& d = c->side[j];
    if (d.tr) continue;
    SMR_CUDA(c, cudaStreamCreateWithFlags(&d.tr, cudaStreamNonBlocking));
    SMR_CUDA(c, cudaStreamCreateWithFlags(&d.nr, cudaStreamNonBlocking));
    SMR_CUDA(c, cudaEventCreateWithFlags(&d.ex, cudaEventDisableTiming));
    SMR_CUDA(c, cudaEventCreateWithFlags(&d.enear, cudaEventDisableTiming));
    d.eout.assign(32, nullptr);
    d.etr.assign(32, nullptr);
    for (int s = 0; s < 32; ++s) {
      SMR_CUDA(c, cudaEventCreateWithFlags(&d.eout[s], cudaEventDisableTiming));
      SMR_CUDA(c, cudaEventCreateWithFlags(&d.etr[s], cudaEventDisableTiming));
    }
  }
  return SMR_OK;
}

void free_side(Ctx* c) {
  for (auto& d : c->side) {
    if (d.tr) cudaStreamDestroy(d.tr);
    if (d.nr) cudaStreamDestroy(d.nr);
    if (d.ex) cudaEventDestroy(d.ex);
    if (d.enear) cudaEventDestroy(d.enear);
    for (auto e : d.eout) if (e) cudaEventDestroy(e);
    for (auto e : d.etr) if (e) cudaEventDestroy(e);
  }
  c->side.clear();
}

// The near product of lane j: on the lane's side stream after an event on
// st (x and its FP32 copy ready), with c->near_ev for the receive to wait on;
// on st itself when the product does not overlap.
static int near_step(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st, int j) {
  c->near_ev = nullptr;
  if (!c->overlap || c->prof || j >= (int)c->side.size() || !c->side[j].nr) return run_near(c, R, prec, x, y, st);
  Ctx::Side& d = c->side[j];
  SMR_CUDA(c, cudaEventRecord(d.ex, st));
  SMR_CUDA(c, cudaStreamWaitEvent(d.nr, d.ex, 0));
  int rc = run_near(c, R, prec, x, y, d.nr);
  SMR_CUDA(c, cudaEventRecord(d.enear, d.nr));
  if (rc) {
    SMR_CUDA(c, cudaStreamWaitEvent(st, d.enear, 0));   // joined even on failure
    return rc;
  }
  c->near_ev = d.enear;
  return SMR_OK;
}

// y = Z x for R right-hand sides [N][R].  FP32 products with several
// right-hand sides run column by column on the single right-hand-side kernels
// (16-byte parts, tensor-core aggregation and receive), which are faster per
// column than the batched kernels: x is transposed to [R][N], each column is
// multiplied, and y is transposed back.  The columns are dealt to the lanes
// round-robin; lane j > 0 runs on its own stream, forked from st after the
// transpose and joined before the transpose back, so a graph captured on st
// holds n_lanes independent chains of single-column products.
int run_product(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st) {
  if (!split_columns(c, R, prec)) {
    int rc = ensure_side(c, 1);
    c->cur_side = 0;
    if (!rc) rc = prep_x32(c, R, prec, x, st);
    if (!rc) rc = near_step(c, R, prec, x, y, st, 0);
    if (!rc) rc = run_far(c, R, prec, x, y, true, st);
    c->near_ev = nullptr;
    c->x32_of = nullptr;                        // the FP32 copy lives for one product only
    return rc;
  }
  const int nl = lanes_for(c, R);
  int rc = ensure_split(c, R);
  if (!rc) rc = ensure_lanes(c, nl);
  if (!rc) rc = ensure_side(c, nl);
  if (rc) return rc;
  const long long n = 2LL * c->npsi * c->p;
  double2* xs = c->d_split;
  double2* ys = c->d_split + (size_t)R * n;
  pbeg(c, st, "transpose", -1, 2.0 * n * R * 16, 0.0);
  rc = transpose_c128(c, n, R, x, xs, st);
  pend(c, st);
  if (rc) return rc;
  if (nl > 1) {
    SMR_CUDA(c, cudaEventRecord(c->lane_fork, st));
    for (int j = 1; j < nl; ++j) SMR_CUDA(c, cudaStreamWaitEvent(c->lanes[j].s, c->lane_fork, 0));
  }
  for (int r = 0; r < R && !rc; ++r) {
    const int j = r % nl;
    cudaStream_t sj = j ? c->lanes[j].s : st;
    use_lane(c, j);
    c->cur_side = j;
    rc = prep_x32(c, 1, prec, xs + (size_t)r * n, sj);
    if (!rc) rc = near_step(c, 1, prec, xs + (size_t)r * n, ys + (size_t)r * n, sj, j);
    if (!rc) rc = far_impl<float>(c, 1, xs + (size_t)r * n, ys + (size_t)r * n, true, sj);
    c->near_ev = nullptr;
  }
  use_lane(c, 0);
  c->cur_side = 0;
  c->x32_of = nullptr;
  // every forked lane is joined, also after an error, so that a capture ends cleanly
  for (int j = 1; j < nl; ++j) {
    cudaError_t e = cudaEventRecord(c->lanes[j].ev, c->lanes[j].s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->lanes[j].ev, 0);
    if (e != cudaSuccess && !rc) {
      c->err = std::string("joining column lanes: ") + cudaGetErrorString(e);
      rc = SMR_E_CUDA;
    }
  }
  if (rc) return rc;
  pbeg(c, st, "transpose", -1, 2.0 * n * R * 16, 0.0);
  rc = transpose_c128(c, R, n, ys, y, st);
  pend(c, st);
  return rc;
}

void free_graphs(Ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  c->capture_stream = nullptr;
}

int run_matvec_graph(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st) {
  for (auto& g : c->graphs)
    if (g.x == x && g.y == y && g.R == R && g.prec == prec) {
      SMR_CUDA(c, cudaGraphLaunch(g.exec, st));
      return SMR_OK;
    }
  // allocations happen outside the capture
  const bool split = split_columns(c, R, prec);
  int rc = ensure_spectra(c, split ? 1 : R, prec);
  if (!rc && split) rc = ensure_split(c, R);
  if (!rc && split) rc = ensure_lanes(c, lanes_for(c, R));
  if (!rc) rc = ensure_side(c, split ? lanes_for(c, R) : 1);
  if (rc) return rc;
  if (!c->capture_stream) SMR_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cs = c->capture_stream;
  // order the capture stream after work already queued on the caller's stream
  cudaEvent_t ev;
  SMR_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  SMR_CUDA(c, cudaEventRecord(ev, st));
  SMR_CUDA(c, cudaStreamWaitEvent(cs, ev, 0));
  SMR_CUDA(c, cudaStreamSynchronize(cs));
  cudaEventDestroy(ev);
  std::vector<ProfRec>* prof = c->prof;
  c->prof = nullptr;
  SMR_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  rc = run_product(c, R, prec, x, y, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  c->prof = prof;
  c->x32_of = nullptr;                          // the capture converted nothing
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) {
    c->err = std::string("graph capture: ") + cudaGetErrorString(e);
    return SMR_E_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
    return SMR_E_CUDA;
  }
  if (c->graphs.size() >= 16) {                  // keep a handful of recent products
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back({x, y, R, prec, exec});
  SMR_CUDA(c, cudaGraphLaunch(exec, st));
  return SMR_OK;
}

int run_precond(Ctx* c, int R, int prec, const double2* r, double2* z, cudaStream_t st) {
  if (!c->pinv_ok) {
    c->err = "a self block is singular: the block-diagonal preconditioner is undefined";
    return SMR_E_INVALID_ARG;
  }
  if (prec == SMR_PREC_FP64)
    return bs_impl<double>(c, c->p, R, c->d_pc_ptr, c->d_pc_col, c->d_pc_blk, c->d_Pinv64, r, z, false, st);
  return bs_impl<float>(c, c->p, R, c->d_pc_ptr, c->d_pc_col, c->d_pc_blk, c->d_Pinv32, r, z, false, st);
}

}  // namespace smr
