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
template <int NCP, int RPTM>
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
  // phi pass: NCP column parts cp = cpp + k * cstepp, rows gp, gp + ngp, ...
  const int NP = 2 * nphP;
  const int ngp = NP <= 256 ? 256 / NP : 1;
  const int gp = NP <= 256 ? tid / NP : 0;
  const int cpp = NP <= 256 ? tid % NP : tid, cstepp = NP <= 256 ? NP : 256;
  float4 acc[NCP][RPTM];
#pragma unroll
  for (int k = 0; k < NCP; ++k)
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
    if (gp < ngp) {
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
  if (gp < ngp) {
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

template <int NCP, int RPTM>
int launch_interp2(Ctx* c, const Level& Lc, const Level& Lp, const float2* F, float2* out, cudaStream_t st) {
  const size_t rowb = (size_t)Lc.nph * 32;
  const size_t sm = 128 + 2 * (size_t)Lc.ip2_BR * rowb + (size_t)Lc.ip2_TR * (rowb + 96) + (size_t)Lc.ip2_TR * 48;
  auto k = k_interp2<NCP, RPTM>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, LV_SMEM_MAX);
  k<<<(unsigned)(Lp.nbox * Lc.ip2_nrt), 256, sm, st>>>(
      Lc.nth, Lc.nph, Lp.nth, Lp.nph, Lc.ip2_TR, Lc.ip2_nrt, Lc.ip2_BR, Lc.d_ip2_band, Lp.d_ch_ptr, Lp.d_ch_idx,
      Lp.d_ch_quad, Lc.d_th_pk, Lc.d_th_ws32, Lc.d_ph_src, Lc.d_ph_w32, Lc.d_shift32, F, out, c->tc_spin,
      c->d_tc_err);
  SMR_LAUNCH(c);
  return SMR_OK;
}


// Anterpolation s + 1 -> s (the weighted adjoint of the interpolation, with
// the conjugate shift).  CTA = (child box c, tile of TI child theta rows);
// 256 threads.  The parent rows [lo, hi) the tile's taps read arrive by one
// bulk copy per row into wrap-padded rows Y (one mbarrier); then, all from
// shared memory:
//   Y[tp][jp]  = w_theta,p[tp] conj(shift_q[tp][jp]) in_P[tp][jp]   (in place)
//   Gt[tp][j]  = sum_k pw[j][k] Y[tp][pst[j] + k]                     (phi-transposed)
//   in_c[i][j] += sum_k tw[i][k] Gt[tp_k][j, or j + N/2 if reflected] (theta-transposed)
// PM / TM: the phi / theta slot counts (the widest transposed stencil).
template <int PM, int TM>
__global__ void __launch_bounds__(256, 3) k_anterp2(int nthC, int nphC, int nthP, int nphP, int TI, int nit, int BR,
                                                    int PADL, int YL, const int* __restrict__ parent,
                                                    const int* __restrict__ quad, const int* __restrict__ lohi,
                                                    const int* __restrict__ pst, const float* __restrict__ pw,
                                                    const int* __restrict__ tws, const int* __restrict__ ttp,
                                                    const float* __restrict__ tw, const float* __restrict__ wthp,
                                                    const float2* __restrict__ shift, const float2* __restrict__ inP,
                                                    float2* __restrict__ inC, uint32_t spin, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int c = blockIdx.x / nit, it = blockIdx.x - c * nit;
  const int i0 = it * TI, ni = min(TI, nthC - i0);
  const int lo = lohi[it], nb = lohi[nit + it] - lo;
  const int B = parent[c], q = quad[c];
  const int Kc = nthC * nphC, Kp = nthP * nphP;
  const uint32_t yrowb = (uint32_t)YL * 32u, prowb = (uint32_t)nphP * 32u, growb = (uint32_t)nphC * 32u;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* Y = smem + 128;                                   // [BR][YL]
  unsigned char* Gt = Y + (size_t)BR * yrowb;                      // [BR][nphC]
  int* tt = reinterpret_cast<int*>(Gt + (size_t)BR * growb);       // [TI][TM] band offset | refl << 31
  float2* twp = reinterpret_cast<float2*>(tt + ((TI * TM + 3) & ~3));  // [TI][TM] (w, w), 16-byte aligned
  int* tf = reinterpret_cast<int*>(twp + TI * TM);                 // [TI] band offset of the window, or -1
  if (tid == 0) {
    lv_mbar_init(lv_saddr(&bar[0]), 1);
    lv_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    lv_expect(lv_saddr(&bar[0]), (uint32_t)nb * prowb);
    const float2* src = inP + ((size_t)B * Kp + (size_t)lo * nphP) * 4;
    for (int r = 0; r < nb; ++r)
      lv_copy_tx(lv_saddr(Y + r * yrowb + (uint32_t)PADL * 32u), src + (size_t)r * nphP * 4, prowb,
                 lv_saddr(&bar[0]));
  }
  for (int t = tid; t < ni * TM; t += 256) {
    const int il = t / TM, i = i0 + il;
    const int pk = ttp[(size_t)i0 * TM + t];
    tt[t] = (int)((uint32_t)((pk & 0xffff) - lo) * growb | ((uint32_t)(pk >> 16) << 31));
    const float w = tw[(size_t)i0 * TM + t];
    twp[t] = make_float2(w, w);
    if (t - il * TM == 0) {
      const int ws = tws[i];
      tf[il] = ws >= 0 ? (int)((uint32_t)(ws - lo) * growb) : -1;
    }
  }
  int ok = 1;
  if (tid == 0) ok = lv_mbar_wait(lv_saddr(&bar[0]), 0u, spin);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      lv_mbar_wait(lv_saddr(&bar[0]), 0u, LV_DRAIN);                 // the row copies land first
      atomicExch(err, 1);
    }
    return;
  }
  // ---- Y = w_theta,p conj(shift) in_P, in place, and the wrap padding
  {
    const int NP = 2 * nphP, PADR = YL - PADL - nphP;
    const int ng = NP <= 256 ? 256 / NP : 1, g = NP <= 256 ? tid / NP : 0;
    const int cp0 = NP <= 256 ? tid % NP : tid, cst = NP <= 256 ? NP : 256;
    if (g < ng)
      for (int cp = cp0; cp < NP; cp += cst) {
        const int jp = cp >> 1, h = cp & 1;
        const uint32_t o = (uint32_t)(PADL + jp) * 32u + (uint32_t)h * 16u;
        const int wr = jp < PADR ? nphP : (jp >= nphP - PADL ? -nphP : 0);   // wrap copy, in columns
        const float2* shp = shift + (size_t)q * Kp + (size_t)lo * nphP + jp;
#pragma unroll 2
        for (int r = g; r < nb; r += ng) {
          float4* p = reinterpret_cast<float4*>(Y + r * yrowb + o);
          const float2 sv = shp[(size_t)r * nphP];
          const float w = wthp[lo + r];
          const float4 v = *p;
          const float cr = w * sv.x, ci = w * sv.y;                 // w conj(s) v
          const float4 y = make_float4(fmaf(cr, v.x, ci * v.y), fmaf(cr, v.y, -ci * v.x),
                                       fmaf(cr, v.z, ci * v.w), fmaf(cr, v.w, -ci * v.z));
          *p = y;
          if (wr) *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(p) + wr * 32) = y;
        }
      }
  }
  __syncthreads();
  // ---- Gt = phi-transposed taps (PM consecutive padded columns per child column)
  const int NC = 2 * nphC, half = nphC >> 1;
  const int ngc = NC <= 256 ? 256 / NC : 1, gc = NC <= 256 ? tid / NC : 0;
  const int cpc = NC <= 256 ? tid % NC : tid, cstc = NC <= 256 ? NC : 256;
  if (gc < ngc)
    for (int cp = cpc; cp < NC; cp += cstc) {
      const int j = cp >> 1, h = cp & 1;
      float2 w2[PM];
#pragma unroll
      for (int k = 0; k < PM; ++k) {
        const float w = pw[(size_t)j * PM + k];
        w2[k] = make_float2(w, w);
      }
      const unsigned char* y0 = Y + (uint32_t)(pst[j] + PADL) * 32u + (uint32_t)h * 16u;
      unsigned char* g0 = Gt + (uint32_t)j * 32u + (uint32_t)h * 16u;
      for (int r = gc; r < nb; r += ngc) {
        const unsigned char* yr = y0 + r * yrowb;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < PM; ++k) fma4p(a, w2[k], lds4(yr + 32 * k));
        *reinterpret_cast<float4*>(g0 + r * growb) = a;
      }
    }
  __syncthreads();
  // ---- in_c += theta-transposed taps
  if (gc < ngc)
    for (int cp = cpc; cp < NC; cp += cstc) {
      const int j = cp >> 1, h = cp & 1;
      const int jr = j < half ? j + half : j - half;
      const uint32_t jo = (uint32_t)j * 32u + (uint32_t)h * 16u, jro = (uint32_t)jr * 32u + (uint32_t)h * 16u;
      float4* dst = reinterpret_cast<float4*>(inC + ((size_t)c * Kc + (size_t)i0 * nphC) * 4) + cp;
      for (int il = gc; il < ni; il += ngc) {
        // the incoming value this row adds to is loaded first, so its latency
        // overlaps the taps
        float4* d = dst + (size_t)il * NC;
        float4 cur = *d;
        const float2* wr = twp + il * TM;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        const int f = tf[il];
        if (f >= 0) {
          const unsigned char* p = Gt + (uint32_t)f + jo;
#pragma unroll
          for (int k = 0; k < TM; ++k) fma4p(a, wr[k], lds4(p + k * growb));
        } else {
          const int* tr = tt + il * TM;
#pragma unroll
          for (int k = 0; k < TM; ++k) {
            const int tk = tr[k];
            fma4p(a, wr[k], lds4(Gt + ((uint32_t)tk & 0x7fffffffu) + (tk < 0 ? jro : jo)));
          }
        }
        cur.x += a.x; cur.y += a.y; cur.z += a.z; cur.w += a.w;
        *d = cur;
      }
    }
}

template <int PM, int TM>
int launch_anterp2(Ctx* c, const Level& Lc, const Level& Lp, cudaStream_t st) {
  const int YL = Lp.nph + Lc.an2_PADL + Lc.an2_PADR;
  const size_t sm = 128 + (size_t)Lc.an2_BR * ((size_t)YL * 32 + (size_t)Lc.nph * 32) +
                    (size_t)((Lc.an2_TI * TM + 3) & ~3) * 4 + (size_t)Lc.an2_TI * TM * 8 + (size_t)Lc.an2_TI * 4;
  auto k = k_anterp2<PM, TM>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, LV_SMEM_MAX);
  k<<<(unsigned)(Lc.nbox * Lc.an2_nit), 256, sm, st>>>(
      Lc.nth, Lc.nph, Lp.nth, Lp.nph, Lc.an2_TI, Lc.an2_nit, Lc.an2_BR, Lc.an2_PADL, YL, Lc.d_parent, Lc.d_quad,
      Lc.d_an2_lo, Lc.d_an2_pst, Lc.d_an2_pw, Lc.d_an2_tws, Lc.d_an2_ttp, Lc.d_an2_tw, Lc.d_wthp32, Lc.d_shift32,
      (const float2*)Lp.d_in, (float2*)Lc.d_in, c->tc_spin, c->d_tc_err);
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

int run_interp2(Ctx* c, int s, cudaStream_t st) {
  const Level &Lc = c->lev[s], &Lp = c->lev[s + 1];
  const float2* F = (const float2*)Lc.d_out;
  float2* out = (float2*)Lp.d_out;
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
