// Level steps of the FP32 product for one right-hand side with the child
// spectra staged in shared memory by bulk copies: interpolation (Sec. V,
// "4x4 Lagrange", child grid -> parent grid, shift, child sum).
//
// Spectra are [box][theta row][phi column][4 fields] complex FP32, 32 bytes
// per direction, so a theta row of a box is one contiguous run and a band of
// consecutive rows is one bulk copy.  A thread owns one 16-byte part (two
// fields) of a column and keeps it across the rows it computes, so the
// column's offsets and taps are computed once and every read in the loops
// is a shared-memory read.
//
// Waits on the copies are bounded by the context's polling limit.  A CTA
// whose wait runs out raises the device error flag, waits (with a fixed
// drain bound) for the copies it has issued, and returns without writing.
#include "smr_internal.h"

namespace smr {

namespace {

constexpr uint32_t LV_DRAIN = 1u << 24;        // polls of the drain after a give-up
// one fixed ceiling for the dynamic shared memory of every launch of these
// kernels: a per-launch value would leave a function's limit below the size
// an earlier-captured graph node of the same function requests
constexpr int LV_SMEM_MAX = 200 * 1024;

__device__ __forceinline__ uint32_t lv_saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void lv_mbar_init(uint32_t a, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
__device__ __forceinline__ void lv_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void lv_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool lv_mbar_test(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool lv_mbar_wait(uint32_t a, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (lv_mbar_test(a, parity)) return true;
  return false;
}
// one bulk copy global -> shared completing on the mbarrier (bytes: multiple of 16)
__device__ __forceinline__ void lv_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// one bulk copy global -> shared whose bytes the mbarrier already expects
__device__ __forceinline__ void lv_copy_tx(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void lv_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// a += w * v on the two complex fields of v, as two packed FP32 FMAs
// (w2 = (w, w))
__device__ __forceinline__ void fma4p(float4& a, const float2 w2, const float4 v) {
  const float2 lo = __ffma2_rn(w2, make_float2(v.x, v.y), make_float2(a.x, a.y));
  const float2 hi = __ffma2_rn(w2, make_float2(v.z, v.w), make_float2(a.z, a.w));
  a = make_float4(lo.x, lo.y, hi.x, hi.y);
}
// a += s * v for the two complex fields of v
__device__ __forceinline__ void cfma4(float4& a, const float2 s, const float4 v) {
  a.x = fmaf(s.x, v.x, a.x); a.x = fmaf(-s.y, v.y, a.x);
  a.y = fmaf(s.x, v.y, a.y); a.y = fmaf(s.y, v.x, a.y);
  a.z = fmaf(s.x, v.z, a.z); a.z = fmaf(-s.y, v.w, a.z);
  a.w = fmaf(s.x, v.w, a.w); a.w = fmaf(s.y, v.z, a.w);
}
__device__ __forceinline__ float4 lds4(const unsigned char* p) { return *reinterpret_cast<const float4*>(p); }

// Interpolation s -> s + 1.  CTA = (parent box B, tile of TR parent theta
// rows); 256 threads.  Per child of B, in child order: the band of child
// rows the tile's theta taps read arrives by one bulk copy (two buffers, the
// next child's copy in flight during this child's passes); theta pass
// G[tr][j] = sum_a w_a band[row_a][j or j + N/2 when reflected] into shared
// memory; phi pass and shift accumulate parent[tr][jp] += shift *
// sum_b w_b G[tr][j0(jp) - 1 + b] in registers (NCP column parts x RPT rows
// per thread, RPTM the compile-time bound).  Finally the tile is stored.
//
// G rows carry the periodic wrap of the phi grid (padded column p = child
// column p - 1 mod N, p = 0 .. N + 2), so the four phi taps of a parent
// column are four consecutive padded columns.  Rows whose theta taps are not
// reflected through a pole read four consecutive band rows.
//
// PAIR (one column part per thread, NCP = 1): a thread's phi pass produces
// two neighbouring parent columns 2m, 2m + 1 from one window of five padded
// columns (their tap windows start at the same column or one apart, the
// parent grid being the finer one), five loads for two outputs instead of
// eight.
template <int NCP, int RPTM, bool PAIR = false>
__global__ void __launch_bounds__(256, 4) k_interp2(int nthC, int nphC, int nthP, int nphP, int TR, int nrt, int BR,
                                                    const int* __restrict__ band, const int* __restrict__ ch_ptr,
                                                    const int* __restrict__ ch_idx, const int* __restrict__ ch_quad,
                                                    const int* __restrict__ th_pk, const float* __restrict__ th_w,
                                                    const int* __restrict__ ph_src, const float* __restrict__ ph_w,
                                                    const float2* __restrict__ shift, const float2* __restrict__ F,
                                                    float2* __restrict__ out, uint32_t spin, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int B = blockIdx.x / nrt, rt = blockIdx.x - B * nrt;
  const int tp0 = rt * TR, ntr = min(TR, nthP - tp0);
  const int r0 = band[rt], nr = band[nrt + rt];
  const uint32_t rowb = (uint32_t)nphC * 32u;                 // bytes of one child theta row
  const uint32_t growb = rowb + 96u;                           // one padded G row
  const uint32_t bandb = (uint32_t)BR * rowb;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);          // [2]
  unsigned char* bufs = smem + 128;                           // [2][BR rows]
  unsigned char* G = bufs + 2 * bandb;                        // [TR][N + 3] directions
  int* tap = reinterpret_cast<int*>(G + (size_t)TR * growb);  // [TR][4]: band byte offset | refl << 31
  float2* tw = reinterpret_cast<float2*>(tap + 4 * TR);       // [TR][4] weights as (w, w)
  const int e0 = ch_ptr[B], nch = ch_ptr[B + 1] - e0;
  const int Kc = nthC * nphC, Kp = nthP * nphP;
  const uint32_t bytes = (uint32_t)nr * rowb;
  if (tid == 0) {
    lv_mbar_init(lv_saddr(&bar[0]), 1);
    lv_mbar_init(lv_saddr(&bar[1]), 1);
    lv_fence_init();
  }
  __syncthreads();
  int issued = 0;                                             // copies issued (thread 0)
  if (tid == 0) {
    for (; issued < 2 && issued < nch; ++issued)
      lv_copy(lv_saddr(bufs + issued * bandb), F + ((size_t)ch_idx[e0 + issued] * Kc + (size_t)r0 * nphC) * 4,
              bytes, lv_saddr(&bar[issued]));
  }
  for (int t = tid; t < 4 * ntr; t += 256) {
    const int pk = th_pk[tp0 * 4 + t];
    tap[t] = (int)((uint32_t)((pk & 0xffff) - r0) * rowb | ((uint32_t)(pk >> 16) << 31));
    const float w = th_w[tp0 * 4 + t];
    tw[t] = make_float2(w, w);
  }
  // theta pass: column part cp = (j, h) fixed per thread, rows g, g + ng, ...
  const int NC = 2 * nphC, half = nphC >> 1;
  const int ngt = NC <= 256 ? 256 / NC : 1;
  const int gt = NC <= 256 ? tid / NC : 0;
  const int cpt = NC <= 256 ? tid % NC : tid, cstept = NC <= 256 ? NC : 256;
  // phi pass: NCP column parts cp = cpp + k * cstepp, rows gp, gp + ngp, ...;
  // with PAIR, (column pair, part) units u = tid % nphP, rows gp, gp + ngp, ...
  const int NP = 2 * nphP;
  const int UN = PAIR ? nphP : NP;
  const int ngp = UN <= 256 ? 256 / UN : 1;
  const int gp = UN <= 256 ? tid / UN : 0;
  const int cpp = UN <= 256 ? tid % UN : tid, cstepp = UN <= 256 ? UN : 256;
  constexpr int NA = PAIR ? 2 : NCP;
  float4 acc[NA][RPTM];
#pragma unroll
  for (int k = 0; k < NA; ++k)
#pragma unroll
    for (int r = 0; r < RPTM; ++r) acc[k][r] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  bool bad = false;
  int e = 0;
  for (; e < nch; ++e) {
    const int b = e & 1;
    // one thread waits for the band; the barrier hands the data to the others
    int ok = 1;
    if (tid == 0) ok = lv_mbar_wait(lv_saddr(&bar[b]), (uint32_t)(e >> 1) & 1u, spin);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    const unsigned char* bd = bufs + b * bandb;
    if (gt < ngt) {
      for (int cp = cpt; cp < NC; cp += cstept) {
        const int j = cp >> 1, h = cp & 1;
        const int jr = j < half ? j + half : j - half;
        const uint32_t jo = (uint32_t)j * 32u + (uint32_t)h * 16u, jro = (uint32_t)jr * 32u + (uint32_t)h * 16u;
        unsigned char* gcol = G + jo + 32u;                   // padded column j + 1
        // columns that also fill the wrap padding: N - 1 -> 0, 0 -> N + 1, 1 -> N + 2
        const int wrap = j == nphC - 1 ? -(int)rowb : (j <= 1 ? (int)rowb : 0);
        for (int tr = gt; tr < ntr; tr += ngt) {
          const int4 tk = *reinterpret_cast<const int4*>(tap + 4 * tr);
          const float4 w01 = *reinterpret_cast<const float4*>(tw + 4 * tr);
          const float4 w23 = *reinterpret_cast<const float4*>(tw + 4 * tr + 2);
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
          if ((tk.x | tk.y | tk.z | tk.w) >= 0) {
            // four consecutive band rows
            const unsigned char* p = bd + (uint32_t)tk.x + jo;
            fma4p(a, make_float2(w01.x, w01.y), lds4(p));
            fma4p(a, make_float2(w01.z, w01.w), lds4(p + rowb));
            fma4p(a, make_float2(w23.x, w23.y), lds4(p + 2 * rowb));
            fma4p(a, make_float2(w23.z, w23.w), lds4(p + 3 * rowb));
          } else {
            fma4p(a, make_float2(w01.x, w01.y), lds4(bd + ((uint32_t)tk.x & 0x7fffffffu) + (tk.x < 0 ? jro : jo)));
            fma4p(a, make_float2(w01.z, w01.w), lds4(bd + ((uint32_t)tk.y & 0x7fffffffu) + (tk.y < 0 ? jro : jo)));
            fma4p(a, make_float2(w23.x, w23.y), lds4(bd + ((uint32_t)tk.z & 0x7fffffffu) + (tk.z < 0 ? jro : jo)));
            fma4p(a, make_float2(w23.z, w23.w), lds4(bd + ((uint32_t)tk.w & 0x7fffffffu) + (tk.w < 0 ? jro : jo)));
          }
          unsigned char* gp_ = gcol + (uint32_t)tr * growb;
          *reinterpret_cast<float4*>(gp_) = a;
          if (wrap) *reinterpret_cast<float4*>(gp_ + wrap) = a;
        }
      }
    }
    __syncthreads();                                          // band b read, G written
    if (tid == 0 && issued < nch) {
      lv_fence_async();
      lv_copy(lv_saddr(bufs + b * bandb), F + ((size_t)ch_idx[e0 + issued] * Kc + (size_t)r0 * nphC) * 4, bytes,
              lv_saddr(&bar[b]));
      ++issued;
    }
    const float2* sh = shift + (size_t)ch_quad[e0 + e] * Kp + (size_t)tp0 * nphP;
    if (PAIR && gp < ngp) {
      const int m = cpp >> 1, h = cpp & 1;
      const int jpa = 2 * m, jpb = jpa + 1;
      const int j0 = ph_src[4 * jpa + 1];
      const bool d1 = ph_src[4 * jpb + 1] != j0;
      const float4 wa = *reinterpret_cast<const float4*>(ph_w + 4 * jpa);
      const float4 wb = *reinterpret_cast<const float4*>(ph_w + 4 * jpb);
      const float2 a0 = make_float2(wa.x, wa.x), a1 = make_float2(wa.y, wa.y);
      const float2 a2 = make_float2(wa.z, wa.z), a3 = make_float2(wa.w, wa.w);
      // column b's four weights over the five-column window
      const float b0s = d1 ? 0.f : wb.x, b1s = d1 ? wb.x : wb.y, b2s = d1 ? wb.y : wb.z;
      const float b3s = d1 ? wb.z : wb.w, b4s = d1 ? wb.w : 0.f;
      const float2 b0 = make_float2(b0s, b0s), b1 = make_float2(b1s, b1s), b2 = make_float2(b2s, b2s);
      const float2 b3 = make_float2(b3s, b3s), b4 = make_float2(b4s, b4s);
      const unsigned char* g0 = G + (uint32_t)j0 * 32u + (uint32_t)h * 16u;
#pragma unroll
      for (int r = 0; r < RPTM; ++r) {
        const int tr = gp + r * ngp;
        if (tr < ntr) {
          const unsigned char* gr = g0 + (uint32_t)tr * growb;
          const float4 v0 = lds4(gr), v1 = lds4(gr + 32), v2 = lds4(gr + 64), v3 = lds4(gr + 96),
                       v4 = lds4(gr + 128);
          float4 sa = make_float4(0.f, 0.f, 0.f, 0.f), sb = sa;
          fma4p(sa, a0, v0); fma4p(sa, a1, v1); fma4p(sa, a2, v2); fma4p(sa, a3, v3);
          fma4p(sb, b0, v0); fma4p(sb, b1, v1); fma4p(sb, b2, v2); fma4p(sb, b3, v3); fma4p(sb, b4, v4);
          const float4 s2 = *reinterpret_cast<const float4*>(sh + (size_t)tr * nphP + jpa);
          cfma4(acc[0][r], make_float2(s2.x, s2.y), sa);
          cfma4(acc[1][r], make_float2(s2.z, s2.w), sb);
        }
      }
    }
    if (!PAIR && gp < ngp) {
#pragma unroll
      for (int k = 0; k < NCP; ++k) {
        const int cp = cpp + k * cstepp;
        if (cp < NP) {
          const int jp = cp >> 1, h = cp & 1;
          // taps: padded columns j0(jp) .. j0(jp) + 3, j0 = ph_src[4 jp + 1]
          const int j0 = ph_src[4 * jp + 1];
          const float4 w = *reinterpret_cast<const float4*>(ph_w + 4 * jp);
          const float2 w0 = make_float2(w.x, w.x), w1 = make_float2(w.y, w.y);
          const float2 w2 = make_float2(w.z, w.z), w3 = make_float2(w.w, w.w);
          const unsigned char* g0 = G + (uint32_t)j0 * 32u + (uint32_t)h * 16u;
          const float2* shp = sh + jp;
#pragma unroll
          for (int r = 0; r < RPTM; ++r) {
            const int tr = gp + r * ngp;
            if (tr < ntr) {
              const unsigned char* gr = g0 + (uint32_t)tr * growb;
              float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
              fma4p(s, w0, lds4(gr));
              fma4p(s, w1, lds4(gr + 32));
              fma4p(s, w2, lds4(gr + 64));
              fma4p(s, w3, lds4(gr + 96));
              cfma4(acc[k][r], shp[(size_t)tr * nphP], s);
            }
          }
        }
      }
    }
    __syncthreads();                                          // G read
  }
  if (bad) {
    if (tid == 0) {
      // drain: every copy issued and not yet consumed lands before the CTA exits
      for (int q = e; q < issued; ++q) lv_mbar_wait(lv_saddr(&bar[q & 1]), (uint32_t)(q >> 1) & 1u, LV_DRAIN);
      atomicExch(err, 1);
    }
    return;
  }
  if (PAIR && gp < ngp) {
    float4* dst = reinterpret_cast<float4*>(out + ((size_t)B * Kp + (size_t)tp0 * nphP) * 4);
    const int m = cpp >> 1, h = cpp & 1;
#pragma unroll
    for (int r = 0; r < RPTM; ++r) {
      const int tr = gp + r * ngp;
      if (tr < ntr) {
        dst[(size_t)tr * NP + 4 * m + h] = acc[0][r];
        dst[(size_t)tr * NP + 4 * m + 2 + h] = acc[1][r];
      }
    }
  }
  if (!PAIR && gp < ngp) {
    float4* dst = reinterpret_cast<float4*>(out + ((size_t)B * Kp + (size_t)tp0 * nphP) * 4);
#pragma unroll
    for (int k = 0; k < NCP; ++k) {
      const int cp = cpp + k * cstepp;
      if (cp < NP) {
#pragma unroll
        for (int r = 0; r < RPTM; ++r) {
          const int tr = gp + r * ngp;
          if (tr < ntr) dst[(size_t)tr * NP + cp] = acc[k][r];
        }
      }
    }
  }
}

template <int NCP, int RPTM, bool PAIR = false>
int launch_interp2(Ctx* c, const Level& Lc, const Level& Lp, const float2* F, float2* out, cudaStream_t st) {
  const size_t rowb = (size_t)Lc.nph * 32;
  const size_t sm = 128 + 2 * (size_t)Lc.ip2_BR * rowb + (size_t)Lc.ip2_TR * (rowb + 96) + (size_t)Lc.ip2_TR * 48;
  auto k = k_interp2<NCP, RPTM, PAIR>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, LV_SMEM_MAX);
  k<<<(unsigned)(Lp.nbox * Lc.ip2_nrt), 256, sm, st>>>(
      Lc.nth, Lc.nph, Lp.nth, Lp.nph, Lc.ip2_TR, Lc.ip2_nrt, Lc.ip2_BR, Lc.d_ip2_band, Lp.d_ch_ptr, Lp.d_ch_idx,
      Lp.d_ch_quad, Lc.d_th_pk, Lc.d_th_ws32, Lc.d_ph_src, Lc.d_ph_w32, Lc.d_shift32, F, out, c->tc_spin,
      c->d_tc_err);
  SMR_LAUNCH(c);
  return SMR_OK;
}


// Anterpolation s + 1 -> s (the weighted adjoint of the interpolation, with
// the conjugate shift).  CTA = (parent box B, tile of TI child theta rows);
// 256 threads.  The parent rows [lo, hi) the tile's taps read arrive by one
// bulk copy (one mbarrier) and serve the four children of B in turn; per
// child c (quadrant q), all from shared memory:
//   Y[tp][jp]  = w_theta,p[tp] conj(shift_q[tp][jp]) in_P[tp][jp]    (wrap-padded rows)
//   Gt[tp][j]  = sum_k pw[j][k] Y[tp][pst[j] + k]                      (phi-transposed)
//   in_c[i][j] += sum_k tw[i][k] Gt[tp_k][j, or j + N/2 if reflected]  (theta-transposed)
// Both transposed passes give a thread two neighbouring outputs from one
// window of loaded values.  PM / TM: the widest phi / theta transposed stencil.
template <int PM, int TM>
__global__ void __launch_bounds__(256, 3) k_anterp2(int nthC, int nphC, int nthP, int nphP, int TI, int nit, int BR,
                                                    int PADL, int YL, const int* __restrict__ ch_ptr,
                                                    const int* __restrict__ ch_idx, const int* __restrict__ ch_quad,
                                                    const int* __restrict__ lohi, const int* __restrict__ ttp,
                                                    const float* __restrict__ tw, const int* __restrict__ pst2,
                                                    const float* __restrict__ pwp, const int* __restrict__ tq,
                                                    const float* __restrict__ twq, const float* __restrict__ wthp,
                                                    const float2* __restrict__ shift, const float2* __restrict__ inP,
                                                    float2* __restrict__ inC, uint32_t spin, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int B = blockIdx.x / nit, it = blockIdx.x - B * nit;
  const int i0 = it * TI, ni = min(TI, nthC - i0);
  const int lo = lohi[it], nb = lohi[nit + it] - lo;
  const int Kc = nthC * nphC, Kp = nthP * nphP;
  const uint32_t yrowb = (uint32_t)YL * 32u, prowb = (uint32_t)nphP * 32u, growb = (uint32_t)nphC * 32u;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* Bd = smem + 128;                                  // [BR][nphP] the parent band
  unsigned char* Y = Bd + (size_t)BR * prowb;                      // [BR][YL]
  unsigned char* Gt = Y + (size_t)BR * yrowb;                      // [BR][nphC]
  int* tt = reinterpret_cast<int*>(Gt + (size_t)BR * growb);       // [TI][TM] band offset | refl << 31
  float2* twp = reinterpret_cast<float2*>(tt + ((TI * TM + 3) & ~3));  // [TI][TM] (w, w), 16-byte aligned
  const int e0 = ch_ptr[B], nch = ch_ptr[B + 1] - e0;
  if (tid == 0) {
    lv_mbar_init(lv_saddr(&bar[0]), 1);
    lv_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    // the band's rows are contiguous in in_P: one copy
    lv_copy(lv_saddr(Bd), inP + ((size_t)B * Kp + (size_t)lo * nphP) * 4, (uint32_t)nb * prowb,
            lv_saddr(&bar[0]));
  }
  // packed theta taps of the tile's rows (used by the row pairs at the poles)
  for (int t = tid; t < ni * TM; t += 256) {
    const int pk = ttp[(size_t)i0 * TM + t];
    tt[t] = (int)((uint32_t)((pk & 0xffff) - lo) * growb | ((uint32_t)(pk >> 16) << 31));
    const float w = tw[(size_t)i0 * TM + t];
    twp[t] = make_float2(w, w);
  }
  int ok = 1;
  if (tid == 0) ok = lv_mbar_wait(lv_saddr(&bar[0]), 0u, spin);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      lv_mbar_wait(lv_saddr(&bar[0]), 0u, LV_DRAIN);                 // the copy lands first
      atomicExch(err, 1);
    }
    return;
  }
  constexpr int WPM = PM + 2, WPS = (WPM + 3) & ~3, WTM = TM + 3, WTS = (WTM + 3) & ~3;
  const int NP = 2 * nphP, PADR = YL - PADL - nphP;
  const int NC = 2 * nphC, half = nphC >> 1;
  for (int e = 0; e < nch; ++e) {
    const int c = ch_idx[e0 + e], q = ch_quad[e0 + e];
    // ---- Y = w_theta,p conj(shift_q) in_P and the wrap padding
    {
      const int ng = NP <= 256 ? 256 / NP : 1, g = NP <= 256 ? tid / NP : 0;
      const int cp0 = NP <= 256 ? tid % NP : tid, cst = NP <= 256 ? NP : 256;
      if (g < ng)
        for (int cp = cp0; cp < NP; cp += cst) {
          const int jp = cp >> 1, h = cp & 1;
          const uint32_t ob = (uint32_t)jp * 32u + (uint32_t)h * 16u;
          const uint32_t oy = (uint32_t)(PADL + jp) * 32u + (uint32_t)h * 16u;
          const int wr = jp < PADR ? nphP : (jp >= nphP - PADL ? -nphP : 0);   // wrap copy, in columns
          const float2* shp = shift + (size_t)q * Kp + (size_t)lo * nphP + jp;
#pragma unroll 2
          for (int r = g; r < nb; r += ng) {
            const float2 sv = shp[(size_t)r * nphP];
            const float w = wthp[lo + r];
            const float4 v = lds4(Bd + r * prowb + ob);
            const float cr = w * sv.x, ci = w * sv.y;               // w conj(s) v
            const float4 y = make_float4(fmaf(cr, v.x, ci * v.y), fmaf(cr, v.y, -ci * v.x),
                                         fmaf(cr, v.z, ci * v.w), fmaf(cr, v.w, -ci * v.z));
            unsigned char* p = Y + r * yrowb + oy;
            *reinterpret_cast<float4*>(p) = y;
            if (wr) *reinterpret_cast<float4*>(p + wr * 32) = y;
          }
        }
    }
    __syncthreads();
    // ---- Gt = phi-transposed taps.  A thread owns a pair of neighbouring
    // child columns (2P, 2P + 1) and one 16-byte part: one window of WPM
    // padded parent columns serves both outputs (dense weights in registers)
    {
      const int NC2 = nphC;                                        // (pair, part) tasks per row
      const int ng2 = NC2 <= 256 ? 256 / NC2 : 1, g2 = NC2 <= 256 ? tid / NC2 : 0;
      const int cp2 = NC2 <= 256 ? tid % NC2 : tid, cs2 = NC2 <= 256 ? NC2 : 256;
      if (g2 < ng2)
        for (int cp = cp2; cp < NC2; cp += cs2) {
          const int P = cp >> 1, h = cp & 1;
          float wa[WPM], wb[WPM];
#pragma unroll
          for (int k = 0; k < WPM; ++k) {
            wa[k] = pwp[((size_t)P * 2 + 0) * WPS + k];
            wb[k] = pwp[((size_t)P * 2 + 1) * WPS + k];
          }
          const unsigned char* y0 = Y + (uint32_t)(pst2[P] + PADL) * 32u + (uint32_t)h * 16u;
          unsigned char* g0 = Gt + (uint32_t)(2 * P) * 32u + (uint32_t)h * 16u;
          for (int r = g2; r < nb; r += ng2) {
            const unsigned char* yr = y0 + r * yrowb;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
#pragma unroll
            for (int k = 0; k < WPM; ++k) {
              const float4 v = lds4(yr + 32 * k);
              a.x = fmaf(wa[k], v.x, a.x); a.y = fmaf(wa[k], v.y, a.y);
              a.z = fmaf(wa[k], v.z, a.z); a.w = fmaf(wa[k], v.w, a.w);
              b.x = fmaf(wb[k], v.x, b.x); b.y = fmaf(wb[k], v.y, b.y);
              b.z = fmaf(wb[k], v.z, b.z); b.w = fmaf(wb[k], v.w, b.w);
            }
            *reinterpret_cast<float4*>(g0 + r * growb) = a;
            *reinterpret_cast<float4*>(g0 + r * growb + 32) = b;
          }
        }
    }
    __syncthreads();
    // ---- in_c += theta-transposed taps.  Task = (pair of child rows, column
    // part), column parts fastest so a warp shares its row pair: one window of
    // WTM consecutive parent rows serves both rows; a pair that reaches a pole
    // takes the packed taps row by row
    {
      const int nq = (ni + 1) >> 1, Q0 = i0 >> 1;
      float4* dst0 = reinterpret_cast<float4*>(inC + ((size_t)c * Kc + (size_t)i0 * nphC) * 4);
      for (int u = tid; u < nq * NC; u += 256) {
        const int qq = u / NC, cp = u - qq * NC;
        const int j = cp >> 1, h = cp & 1;
        const uint32_t jo = (uint32_t)j * 32u + (uint32_t)h * 16u;
        const int il0 = 2 * qq, two = il0 + 1 < ni;
        float4* d0 = dst0 + (size_t)il0 * NC + cp;
        // the incoming values these rows add to are loaded first
        float4 cur0 = *d0, cur1 = two ? d0[NC] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        const int ws = tq[Q0 + qq];
        if (ws >= 0) {
          const unsigned char* p = Gt + (uint32_t)(ws - lo) * growb + jo;
          const float4* w0 = reinterpret_cast<const float4*>(twq + (size_t)(Q0 + qq) * 2 * WTS);
          const float4* w1 = w0 + WTS / 4;
          float wa[WTS], wb[WTS];
#pragma unroll
          for (int k = 0; k < WTS / 4; ++k) {
            const float4 x = __ldg(w0 + k), y = __ldg(w1 + k);
            wa[4 * k] = x.x; wa[4 * k + 1] = x.y; wa[4 * k + 2] = x.z; wa[4 * k + 3] = x.w;
            wb[4 * k] = y.x; wb[4 * k + 1] = y.y; wb[4 * k + 2] = y.z; wb[4 * k + 3] = y.w;
          }
#pragma unroll
          for (int k = 0; k < WTM; ++k) {
            const float4 v = lds4(p + k * growb);
            a.x = fmaf(wa[k], v.x, a.x); a.y = fmaf(wa[k], v.y, a.y);
            a.z = fmaf(wa[k], v.z, a.z); a.w = fmaf(wa[k], v.w, a.w);
            b.x = fmaf(wb[k], v.x, b.x); b.y = fmaf(wb[k], v.y, b.y);
            b.z = fmaf(wb[k], v.z, b.z); b.w = fmaf(wb[k], v.w, b.w);
          }
        } else {
          const int jr = j < half ? j + half : j - half;
          const uint32_t jro = (uint32_t)jr * 32u + (uint32_t)h * 16u;
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            if (rr == 1 && !two) break;
            const int* tr = tt + (il0 + rr) * TM;
            const float2* wr = twp + (il0 + rr) * TM;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < TM; ++k) {
              const int tk = tr[k];
              fma4p(acc, wr[k], lds4(Gt + ((uint32_t)tk & 0x7fffffffu) + (tk < 0 ? jro : jo)));
            }
            if (rr == 0) a = acc; else b = acc;
          }
        }
        cur0.x += a.x; cur0.y += a.y; cur0.z += a.z; cur0.w += a.w;
        *d0 = cur0;
        if (two) {
          cur1.x += b.x; cur1.y += b.y; cur1.z += b.z; cur1.w += b.w;
          d0[NC] = cur1;
        }
      }
    }
    __syncthreads();                                               // Y and Gt free for the next child
  }
}

template <int PM, int TM>
int launch_anterp2(Ctx* c, const Level& Lc, const Level& Lp, cudaStream_t st) {
  const int YL = Lp.nph + Lc.an2_PADL + Lc.an2_PADR;
  const size_t sm = 128 + (size_t)Lc.an2_BR * ((size_t)Lp.nph * 32 + (size_t)YL * 32 + (size_t)Lc.nph * 32) +
                    (size_t)((Lc.an2_TI * TM + 3) & ~3) * 4 + (size_t)Lc.an2_TI * TM * 8;
  auto k = k_anterp2<PM, TM>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, LV_SMEM_MAX);
  k<<<(unsigned)(Lp.nbox * Lc.an2_nit), 256, sm, st>>>(
      Lc.nth, Lc.nph, Lp.nth, Lp.nph, Lc.an2_TI, Lc.an2_nit, Lc.an2_BR, Lc.an2_PADL, YL, Lp.d_ch_ptr, Lp.d_ch_idx,
      Lp.d_ch_quad, Lc.d_an2_lo, Lc.d_an2_ttp, Lc.d_an2_tw, Lc.d_an2_pst2, Lc.d_an2_pwp, Lc.d_an2_tq, Lc.d_an2_twq,
      Lc.d_wthp32, Lc.d_shift32, (const float2*)Lp.d_in, (float2*)Lc.d_in, c->tc_spin, c->d_tc_err);
  SMR_LAUNCH(c);
  return SMR_OK;
}


}  // namespace

bool interp2_ok(const Ctx* c, int s) {
  const Level& Lc = c->lev[s];
  const size_t rowb = (size_t)Lc.nph * 32;
  const size_t sm = 128 + 2 * (size_t)Lc.ip2_BR * rowb + (size_t)Lc.ip2_TR * (rowb + 96) + (size_t)Lc.ip2_TR * 48;
  return c->lv2_enable && c->d_tc_err && Lc.ip2_NCP >= 1 && Lc.ip2_NCP <= 5 && sm <= (size_t)LV_SMEM_MAX &&
         Lc.ip2_RPT <= (Lc.ip2_NCP == 1 ? 6 : 8 / Lc.ip2_NCP);
}

// The paired phi pass: one column part per thread, at most three rows per
// thread in the paired layout, and every pair's tap windows one column apart
// at most (checked when the tables are built).
bool interp2_pair_ok(const Ctx* c, int s) {
  const Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
  if (Lc.ip2_NCP != 1 || !Lc.ip2_pair || Lp.nph > 256 || (Lp.nph & 1)) return false;
  const int ngq = 256 / Lp.nph;
  return (Lc.ip2_TR + ngq - 1) / ngq <= 3;
}

int run_interp2(Ctx* c, int s, cudaStream_t st) {
  const Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
  const float2* F = (const float2*)Lc.d_out;
  float2* out = (float2*)Lp.d_out;
  if (Lc.tune_ip[1] == 3 && interp2_pair_ok(c, s)) return launch_interp2<1, 3, true>(c, Lc, Lp, F, out, st);
  switch (Lc.ip2_NCP) {
    case 1: return launch_interp2<1, 6>(c, Lc, Lp, F, out, st);
    case 2: return launch_interp2<2, 4>(c, Lc, Lp, F, out, st);
    case 3: return launch_interp2<3, 2>(c, Lc, Lp, F, out, st);
    case 4: return launch_interp2<4, 2>(c, Lc, Lp, F, out, st);
    case 5: return launch_interp2<5, 1>(c, Lc, Lp, F, out, st);
    default: c->err = "interpolation tile shape"; return SMR_E_INVALID_ARG;
  }
}

}  // namespace smr

namespace smr {
bool anterp2_ok(const Ctx* c, int s) {
  const Level& Lc = c->lev[s];
  return c->lv2_enable && c->d_tc_err && Lc.an2_TI > 0 && (Lc.an2_PM == 7 || Lc.an2_PM == 8) &&
         (Lc.an2_TM == 7 || Lc.an2_TM == 8);
}

int run_anterp2(Ctx* c, int s, cudaStream_t st) {
  const Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
  if (Lc.an2_PM == 7) return Lc.an2_TM == 7 ? launch_anterp2<7, 7>(c, Lc, Lp, st) : launch_anterp2<7, 8>(c, Lc, Lp, st);
  return Lc.an2_TM == 7 ? launch_anterp2<8, 7>(c, Lc, Lp, st) : launch_anterp2<8, 8>(c, Lc, Lp, st);
}
}  // namespace smr
