// C ABI of libsmr (declared in include/smr.h): context, scene setup and the
// entry points.  Scene setup builds the quadtree of Sec. IV (each particle its
// own finest group, parents = 2x2 children), the interaction lists, the
// k-space grids of Sec. V, the 4x4 Lagrange interpolation taps and their
// weighted adjoint, and then calls the FP64 table generators on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "smr_internal.h"

using namespace smr;

namespace {

const double PI = 3.14159265358979323846;

int fail(Ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

template <typename T> void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_scene(Ctx* c) {
  free_graphs(c);
  free_lanes(c);
  for (auto& L : c->lev) {
    dfree(L.d_khat); dfree(L.d_w); dfree(L.d_il_ptr); dfree(L.d_il_src); dfree(L.d_il_off); dfree(L.d_il_pk);
    dfree(L.d_T64); dfree(L.d_T32); dfree(L.d_parent); dfree(L.d_quad); dfree(L.d_ch_ptr);
    dfree(L.d_ch_idx); dfree(L.d_ch_quad); dfree(L.d_th_src); dfree(L.d_th_refl); dfree(L.d_th_w64);
    dfree(L.d_th_w32); dfree(L.d_th_pk); dfree(L.d_th_ws64); dfree(L.d_th_ws32); dfree(L.d_ph_src); dfree(L.d_ph_w64); dfree(L.d_ph_w32); dfree(L.d_shift64);
    dfree(L.d_shift32); dfree(L.d_shift4_32); dfree(L.d_ip2_band); dfree(L.d_an2_lo);
    dfree(L.d_an2_ttp); dfree(L.d_an2_tw); dfree(L.d_an2_pst2); dfree(L.d_an2_pwp);
    dfree(L.d_an2_tq); dfree(L.d_an2_twq); dfree(L.d_ant_lo); dfree(L.d_ant_pjp); dfree(L.d_ant_pw64); dfree(L.d_ant_pw32);
    dfree(L.d_ant_ttp); dfree(L.d_ant_tw64); dfree(L.d_ant_tw32);
    dfree(L.d_tht_ptr); dfree(L.d_tht_tp); dfree(L.d_tht_refl); dfree(L.d_tht_w64); dfree(L.d_tht_w32);
    dfree(L.d_pht_ptr); dfree(L.d_pht_jp); dfree(L.d_pht_w64); dfree(L.d_pht_w32); dfree(L.d_wthp64);
    dfree(L.d_wthp32); dfree(L.d_boxmap); dfree(L.d_offid); dfree(L.d_tiles); dfree(L.d_tiles8);
    for (int q = 0; q < 2; ++q) {
      if (L.buf_out[q]) cudaFree(L.buf_out[q]);
      if (L.buf_in[q]) cudaFree(L.buf_in[q]);
      L.buf_out[q] = L.buf_in[q] = nullptr;
    }
    L.d_out = L.d_in = nullptr;
  }
  c->lev.clear();
  dfree(c->d_modes); dfree(c->d_rq); dfree(c->d_P64); dfree(c->d_P32); dfree(c->d_sid);
  dfree(c->d_centres); dfree(c->d_dshift); dfree(c->d_nr_ptr); dfree(c->d_nr_col); dfree(c->d_nr_blk);
  dfree(c->d_cell_of); dfree(c->d_cell_ptr); dfree(c->d_cell_idx);
  for (int q = 0; q < 2; ++q) {
    if (c->pspec[q]) cudaFree(c->pspec[q]);
    c->pspec[q] = nullptr;
  }
  c->multi = 0;
  dfree(c->d_B64); dfree(c->d_B32); dfree(c->d_tcn_img); dfree(c->d_tcn_blk); dfree(c->d_tcn_start);
  dfree(c->d_tcn_count); dfree(c->d_tcn_nu); dfree(c->d_tcn_mu); dfree(c->d_x32);
  dfree(c->d_tcn_mask); dfree(c->d_tcn_part); dfree(c->d_Pinv64); dfree(c->d_Pinv32); dfree(c->d_pc_ptr);
  dfree(c->d_pc_col); dfree(c->d_pc_blk); dfree(c->d_tmp);
  dfree(c->d_arr);
  dfree(c->d_tile_shape); dfree(c->d_tile_start); dfree(c->d_tile_count); dfree(c->d_perm);
  dfree(c->d_tc_rec); dfree(c->d_tc_agg); dfree(c->d_tc_perm); dfree(c->d_lpc); dfree(c->d_split);
  dfree(c->d_pcw);
  c->pcw_elems = 0;
  dfree(c->d_polyw);
  c->polyw_elems = 0;
  free_clusters(c);
  c->split_elems = 0;
  c->lpc_ready = false; dfree(c->d_tc_shape); dfree(c->d_tc_start); dfree(c->d_tc_count);
  c->tc_ready = false;
  c->tc_agg_ready = false;
  for (int q = 0; q < 2; ++q) {
    if (c->G_buf[q]) cudaFree(c->G_buf[q]);
    c->G_buf[q] = nullptr;
    c->G_size[q] = 0;
    c->buf_R[q] = 0;
  }
  c->d_G = nullptr;
  c->G_bytes = 0;
  c->tmp_elems = 0;
  c->spec_R = 0;
  c->spec_prec = -1;
  c->have_scene = false;
}

// truncation order at level s (see smr_opts.level_rule)
int truncation(const Ctx* c, int s) {
  if (s == 0) return c->opts.L0;
  if (c->opts.level_rule == SMR_LRULE_DOUBLE) return c->opts.L0 << s;
  double kd = c->k * std::sqrt(2.0) * c->opts.pitch * (double)(1 << s);
  return (int)std::ceil(kd + 1.8 * std::pow(c->opts.digits, 2.0 / 3.0) * std::cbrt(kd));
}

void make_grid(Level& L) {
  std::vector<double> x, w;
  hm::gauss_legendre(L.L + 1, x, w);
  L.nth = L.L + 1;
  L.nph = 2 * L.L + 2;
  L.K = L.nth * L.nph;
  L.khat.resize(3 * (size_t)L.K);
  L.w.resize(L.K);
  for (int i = 0; i < L.nth; ++i) {
    double th = std::acos(x[i]), st = std::sin(th), ct = std::cos(th);
    for (int j = 0; j < L.nph; ++j) {
      double ph = 2.0 * PI * j / L.nph;
      int k = i * L.nph + j;
      L.khat[3 * k] = st * std::cos(ph);
      L.khat[3 * k + 1] = st * std::sin(ph);
      L.khat[3 * k + 2] = ct;
      L.w[k] = w[i] * 2.0 * PI / L.nph;
    }
  }
}

std::vector<double> grid_theta(const Level& L) {
  std::vector<double> x, w, th(L.nth);
  hm::gauss_legendre(L.nth, x, w);
  for (int i = 0; i < L.nth; ++i) th[i] = std::acos(x[i]);
  return th;
}

void lagrange4(const double* nodes, double t, double* out) {
  for (int a = 0; a < 4; ++a) {
    double v = 1.0;
    for (int b = 0; b < 4; ++b)
      if (b != a) v *= (t - nodes[b]) / (nodes[a] - nodes[b]);
    out[a] = v;
  }
}

// 4x4 Lagrange taps from the child grid C to the parent grid P; the stencil
// in theta is reflected through the poles, (-theta, phi) = (theta, phi + pi),
// where both spherical components change sign.
int build_interp(Ctx* c, Level& C, const Level& P) {
  std::vector<double> thc = grid_theta(C), thp = grid_theta(P);
  int ntc = C.nth;
  std::vector<int> tsrc(4 * P.nth), trefl(4 * P.nth), psrc(4 * P.nph);
  std::vector<double> tw(4 * P.nth), pw(4 * P.nph);
  for (int tp = 0; tp < P.nth; ++tp) {
    double t = thp[tp];
    int i0 = (int)(std::upper_bound(thc.begin(), thc.end(), t) - thc.begin()) - 1;
    double nodes[4];
    for (int a = 0; a < 4; ++a) {
      int i = i0 - 1 + a;
      if (i < 0) { nodes[a] = -thc[-1 - i]; tsrc[4 * tp + a] = -1 - i; trefl[4 * tp + a] = 1; }
      else if (i >= ntc) {
        nodes[a] = 2.0 * PI - thc[2 * ntc - 1 - i];
        tsrc[4 * tp + a] = 2 * ntc - 1 - i;
        trefl[4 * tp + a] = 1;
      } else { nodes[a] = thc[i]; tsrc[4 * tp + a] = i; trefl[4 * tp + a] = 0; }
    }
    lagrange4(nodes, t, &tw[4 * tp]);
  }
  double dphi = 2.0 * PI / C.nph;
  for (int jp = 0; jp < P.nph; ++jp) {
    double f = 2.0 * PI * jp / P.nph;
    int j0 = (int)std::floor(f / dphi);
    double nodes[4];
    for (int b = 0; b < 4; ++b) {
      int j = j0 - 1 + b;
      nodes[b] = j * dphi;
      psrc[4 * jp + b] = ((j % C.nph) + C.nph) % C.nph;
    }
    lagrange4(nodes, f, &pw[4 * jp]);
  }
  std::vector<float> tw32(tw.begin(), tw.end()), pw32(pw.begin(), pw.end());
  // single right-hand-side kernel: source row | reflected << 16, and the
  // weights with the reflection's sign folded in
  std::vector<int> tpk(4 * P.nth);
  std::vector<double> tws(4 * P.nth);
  for (int e = 0; e < 4 * P.nth; ++e) {
    tpk[e] = tsrc[e] | (trefl[e] << 16);
    tws[e] = trefl[e] ? -tw[e] : tw[e];
  }
  std::vector<float> tws32(tws.begin(), tws.end());
  int rc;
  if ((rc = upload(c, &C.d_th_pk, tpk)) || (rc = upload(c, &C.d_th_ws64, tws)) ||
      (rc = upload(c, &C.d_th_ws32, tws32)))
    return rc;
  // staged FP32 interpolation (k_interp2): 256 threads; the phi pass gives a
  // thread NCP column parts (16 bytes each, 2 per direction) of RPT rows; a
  // tile of TR parent rows reads the band of child rows its taps name
  {
    const int NP = 2 * P.nph;
    int ng, ncp, rpt;
    if (NP <= 256) { ncp = 1; ng = 256 / NP; rpt = 6; }
    else { ncp = (NP + 255) / 256; ng = 1; rpt = std::max(1, 8 / ncp); }
    int TR = std::min(P.nth, ng * rpt);
    const size_t rowb = (size_t)C.nph * 32;
    auto band_of = [&](int t0, int t1, int* r0, int* nr) {
      int lo = ntc, hi = -1;
      for (int tp = t0; tp < t1; ++tp)
        for (int a = 0; a < 4; ++a) { lo = std::min(lo, tsrc[4 * tp + a]); hi = std::max(hi, tsrc[4 * tp + a]); }
      *r0 = lo;
      *nr = hi - lo + 1;
    };
    // shrink the tile until two bands and the tile's theta-pass rows fit 110 KB
    for (;;) {
      int br = 0;
      for (int t0 = 0; t0 < P.nth; t0 += TR) {
        int r0, nr;
        band_of(t0, std::min(P.nth, t0 + TR), &r0, &nr);
        br = std::max(br, nr);
      }
      if (TR == 1 || 2 * (size_t)br * rowb + (size_t)TR * (rowb + 96) <= 110 * 1024) break;
      TR = std::max(1, TR / 2);
    }
    C.ip2_TR = TR;
    C.ip2_nrt = (P.nth + TR - 1) / TR;
    // paired phi pass: the windows of columns 2m and 2m + 1 start at most one
    // column apart and five padded columns from the first stay in the row
    C.ip2_pair = (P.nph % 2 == 0);
    for (int m = 0; 2 * m + 1 < P.nph && C.ip2_pair; ++m) {
      const int ja = psrc[4 * (2 * m) + 1], jb = psrc[4 * (2 * m + 1) + 1];
      C.ip2_pair = (jb - ja == 0 || jb - ja == 1) && ja <= C.nph - 2;
    }
    C.ip2_NCP = ncp;
    C.ip2_RPT = (TR + ng - 1) / ng;
    std::vector<int> band(2 * C.ip2_nrt);
    C.ip2_BR = 0;
    for (int t = 0; t < C.ip2_nrt; ++t) {
      band_of(t * TR, std::min(P.nth, (t + 1) * TR), &band[t], &band[C.ip2_nrt + t]);
      C.ip2_BR = std::max(C.ip2_BR, band[C.ip2_nrt + t]);
    }
    if ((rc = upload(c, &C.d_ip2_band, band))) return rc;
  }
  if ((rc = upload(c, &C.d_th_src, tsrc)) || (rc = upload(c, &C.d_th_refl, trefl)) ||
      (rc = upload(c, &C.d_th_w64, tw)) || (rc = upload(c, &C.d_th_w32, tw32)) ||
      (rc = upload(c, &C.d_ph_src, psrc)) || (rc = upload(c, &C.d_ph_w64, pw)) ||
      (rc = upload(c, &C.d_ph_w32, pw32)))
    return rc;
  // separable transposes: theta taps grouped by child row (sign and 1/w_theta(child)
  // folded in), phi taps grouped by child column (dphi_p / dphi_c folded in)
  {
    std::vector<double> xc, wc, xp, wpth;
    hm::gauss_legendre(C.nth, xc, wc);
    hm::gauss_legendre(P.nth, xp, wpth);
    std::vector<int> tptr(C.nth + 1, 0), ttp, trf;
    std::vector<double> tww;
    for (int tp = 0; tp < P.nth; ++tp)
      for (int a = 0; a < 4; ++a) tptr[tsrc[4 * tp + a] + 1]++;
    for (int i = 0; i < C.nth; ++i) tptr[i + 1] += tptr[i];
    ttp.resize(tptr[C.nth]); trf.resize(tptr[C.nth]); tww.resize(tptr[C.nth]);
    std::vector<int> tf(tptr.begin(), tptr.end() - 1);
    for (int tp = 0; tp < P.nth; ++tp)
      for (int a = 0; a < 4; ++a) {
        int i = tsrc[4 * tp + a], e = tf[i]++;
        ttp[e] = tp;
        trf[e] = trefl[4 * tp + a];
        tww[e] = (trefl[4 * tp + a] ? -1.0 : 1.0) * tw[4 * tp + a] / wc[i];
      }
    std::vector<int> pptr(C.nph + 1, 0), pjp;
    std::vector<double> pww;
    for (int jp = 0; jp < P.nph; ++jp)
      for (int b = 0; b < 4; ++b) pptr[psrc[4 * jp + b] + 1]++;
    for (int j = 0; j < C.nph; ++j) pptr[j + 1] += pptr[j];
    pjp.resize(pptr[C.nph]); pww.resize(pptr[C.nph]);
    std::vector<int> pf(pptr.begin(), pptr.end() - 1);
    double ratio = (double)C.nph / (double)P.nph;   // dphi_p / dphi_c
    for (int jp = 0; jp < P.nph; ++jp)
      for (int b = 0; b < 4; ++b) {
        int j = psrc[4 * jp + b], e = pf[j]++;
        pjp[e] = jp;
        pww[e] = pw[4 * jp + b] * ratio;
      }
    std::vector<float> tww32(tww.begin(), tww.end()), pww32(pww.begin(), pww.end()),
        wpth32(wpth.begin(), wpth.end());
    if ((rc = upload(c, &C.d_tht_ptr, tptr)) || (rc = upload(c, &C.d_tht_tp, ttp)) ||
        (rc = upload(c, &C.d_tht_refl, trf)) || (rc = upload(c, &C.d_tht_w64, tww)) ||
        (rc = upload(c, &C.d_tht_w32, tww32)) || (rc = upload(c, &C.d_pht_ptr, pptr)) ||
        (rc = upload(c, &C.d_pht_jp, pjp)) || (rc = upload(c, &C.d_pht_w64, pww)) ||
        (rc = upload(c, &C.d_pht_w32, pww32)) || (rc = upload(c, &C.d_wthp64, wpth)) ||
        (rc = upload(c, &C.d_wthp32, wpth32)))
      return rc;
    // tiles of the fused single right-hand-side anterpolation: child theta
    // rows in tiles of TI, each with the range [lo, hi) of parent rows its
    // transposed taps read; GR = the widest range
    C.ant_TI = C.nth <= 24 ? C.nth : 16;
    C.ant_nit = (C.nth + C.ant_TI - 1) / C.ant_TI;
    std::vector<int> lohi(2 * C.ant_nit);
    C.ant_GR = 1;
    for (int it = 0; it < C.ant_nit; ++it) {
      int i0 = it * C.ant_TI, i1 = std::min(C.nth, i0 + C.ant_TI);
      int lo = P.nth, hi = 0;
      for (int e = tptr[i0]; e < tptr[i1]; ++e) {
        lo = std::min(lo, ttp[e]);
        hi = std::max(hi, ttp[e] + 1);
      }
      if (hi <= lo) { lo = 0; hi = 1; }            // no taps: one (zero-weighted) row
      lohi[it] = lo;
      lohi[C.ant_nit + it] = hi;
      C.ant_GR = std::max(C.ant_GR, hi - lo);
    }
    // column chunk per precision: GR x 2 JC directions in 48 KB of shared memory
    for (int q = 0; q < 2; ++q) {
      int dirb = q == 0 ? 64 : 32;                  // SMR_PREC_FP64, SMR_PREC_FP32
      int jc = (48 * 1024) / (C.ant_GR * 2 * dirb);
      C.ant_JC[q] = std::max(1, std::min(C.nph / 2, jc));
    }
    // the per-parent FP32 kernel holds four quadrants' rows: 52 KB for four CTAs per SM
    C.ant_JC5 = std::max(1, std::min(C.nph / 2, (52 * 1024) / (4 * C.ant_GR * 2 * 32)));
    if ((rc = upload(c, &C.d_ant_lo, lohi))) return rc;
    // padded transposed taps
    int pm = 0, tm = 0;
    for (int j = 0; j < C.nph; ++j) pm = std::max(pm, pptr[j + 1] - pptr[j]);
    for (int i = 0; i < C.nth; ++i) tm = std::max(tm, tptr[i + 1] - tptr[i]);
    C.ant_PM = (pm + 3) / 4 * 4;
    C.ant_TM = (tm + 3) / 4 * 4;
    C.ant_PMx = pm;
    C.ant_TMx = tm;
    std::vector<int> ppj((size_t)C.nph * C.ant_PM), tpk((size_t)C.nth * C.ant_TM);
    std::vector<double> ppw((size_t)C.nph * C.ant_PM, 0.0), tpw((size_t)C.nth * C.ant_TM, 0.0);
    for (int j = 0; j < C.nph; ++j)
      for (int q = 0; q < C.ant_PM; ++q) {
        int e = pptr[j] + q;
        bool real = e < pptr[j + 1];
        // padding repeats the column's first tap (or column 0) with weight 0
        ppj[(size_t)j * C.ant_PM + q] = real ? pjp[e] : (pptr[j + 1] > pptr[j] ? pjp[pptr[j]] : 0);
        ppw[(size_t)j * C.ant_PM + q] = real ? pww[e] : 0.0;
      }
    for (int i = 0; i < C.nth; ++i)
      for (int q = 0; q < C.ant_TM; ++q) {
        int e = tptr[i] + q;
        bool real = e < tptr[i + 1];
        // padding repeats the row's first tap (or the tile's first parent row)
        // with weight 0, so that it reads a row the tile computed
        int pk = lohi[i / C.ant_TI];
        if (real) pk = ttp[e] | (trf[e] << 16);
        else if (tptr[i + 1] > tptr[i]) pk = ttp[tptr[i]] | (trf[tptr[i]] << 16);
        tpk[(size_t)i * C.ant_TM + q] = pk;
        tpw[(size_t)i * C.ant_TM + q] = real ? tww[e] : 0.0;
      }
    // staged FP32 anterpolation (k_anterp2)
    {
      const int PM = pm, TM = tm;
      // phi: the taps of child column j are consecutive parent columns (mod
      // nphP); unwrap them around j's position and keep PM slots from the first
      std::vector<int> pst(C.nph);
      std::vector<float> pw2((size_t)C.nph * PM, 0.f);
      int padl = 0, padr = 0;
      for (int j = 0; j < C.nph; ++j) {
        const int ref = (int)std::lround((double)j * P.nph / C.nph);
        int dmin = 1 << 30;
        std::vector<int> dd;
        for (int e = pptr[j]; e < pptr[j + 1]; ++e) {
          int d = ((pjp[e] - ref) % P.nph + P.nph) % P.nph;
          if (d > P.nph / 2) d -= P.nph;
          dd.push_back(d);
          dmin = std::min(dmin, d);
        }
        if (dd.empty()) dmin = 0;
        pst[j] = ref + dmin;
        for (size_t t = 0; t < dd.size(); ++t) {
          const int slot = dd[t] - dmin;
          if (slot >= PM) return fail(c, SMR_E_INVALID_ARG, "anterpolation phi taps are not consecutive");
          pw2[(size_t)j * PM + slot] += (float)pww[pptr[j] + t];
        }
        padl = std::max(padl, -pst[j]);
        padr = std::max(padr, pst[j] + PM - P.nph);
      }
      // theta: consecutive parent rows (no pole reflection) from a window start
      // kept inside [0, nthP - TM]; otherwise the packed taps
      std::vector<int> tws(C.nth), ttp2((size_t)C.nth * TM);
      std::vector<float> tw2((size_t)C.nth * TM, 0.f);
      for (int i = 0; i < C.nth; ++i) {
        bool refl = false;
        int first = P.nth;
        for (int e = tptr[i]; e < tptr[i + 1]; ++e) { refl = refl || trf[e]; first = std::min(first, ttp[e]); }
        if (tptr[i + 1] == tptr[i]) first = 0;
        if (!refl && P.nth >= TM) {
          const int ws = std::min(first, P.nth - TM);
          tws[i] = ws;
          for (int e = tptr[i]; e < tptr[i + 1]; ++e) {
            const int slot = ttp[e] - ws;
            if (slot < 0 || slot >= TM) return fail(c, SMR_E_INVALID_ARG, "anterpolation theta taps are not consecutive");
            tw2[(size_t)i * TM + slot] += (float)tww[e];
          }
          for (int k = 0; k < TM; ++k) ttp2[(size_t)i * TM + k] = ws + k;
        } else {
          tws[i] = -1;
          for (int k = 0; k < TM; ++k) {
            const int e = tptr[i] + k;
            const bool real = e < tptr[i + 1];
            const int e0 = tptr[i + 1] > tptr[i] ? tptr[i] : -1;
            ttp2[(size_t)i * TM + k] = real ? (ttp[e] | (trf[e] << 16)) : (e0 >= 0 ? (ttp[e0] | (trf[e0] << 16)) : 0);
            tw2[(size_t)i * TM + k] = real ? (float)tww[e] : 0.f;
          }
        }
      }
      // pairs of neighbouring child columns (rows) share one window of loaded
      // values: dense weights over PM + 2 parent columns (the second column's
      // taps start 0..2 columns after the first's) and TM + 3 parent rows;
      // weight rows padded to multiples of 4 for 16-byte loads
      const int WPM = PM + 2, WTM = TM + 3, WPS = (WPM + 3) & ~3, WTS = (WTM + 3) & ~3;
      const int npp = C.nph / 2, nqp = (C.nth + 1) / 2;
      std::vector<int> pst2(npp);
      std::vector<float> pwp((size_t)npp * 2 * WPS, 0.f);
      bool pairs_ok = (C.nph % 2) == 0;
      for (int q = 0; q < npp && pairs_ok; ++q) {
        const int ja = 2 * q, jb = 2 * q + 1, d = pst[jb] - pst[ja];
        if (d < 0 || d + PM > WPM) { pairs_ok = false; break; }
        pst2[q] = pst[ja];
        for (int k = 0; k < PM; ++k) {
          pwp[((size_t)q * 2 + 0) * WPS + k] = pw2[(size_t)ja * PM + k];
          pwp[((size_t)q * 2 + 1) * WPS + d + k] = pw2[(size_t)jb * PM + k];
        }
        padl = std::max(padl, -pst2[q]);
        padr = std::max(padr, pst2[q] + WPM - P.nph);
      }
      // row pairs (2q, 2q + 1): window start, or -1 where a row reaches a pole
      std::vector<int> tq(nqp, -1);
      std::vector<float> twq((size_t)nqp * 2 * WTS, 0.f);
      for (int q = 0; q < nqp; ++q) {
        const int ia = 2 * q, ib = 2 * q + 1;
        if (tws[ia] < 0 || (ib < C.nth && tws[ib] < 0) || P.nth < WTM) continue;
        const int ws = std::min(tws[ia], P.nth - WTM);
        const int da = tws[ia] - ws, db = ib < C.nth ? tws[ib] - ws : 0;
        if (da < 0 || da + TM > WTM || db < 0 || db + TM > WTM) continue;
        tq[q] = ws;
        for (int k = 0; k < TM; ++k) {
          twq[((size_t)q * 2 + 0) * WTS + da + k] = tw2[(size_t)ia * TM + k];
          if (ib < C.nth) twq[((size_t)q * 2 + 1) * WTS + db + k] = tw2[(size_t)ib * TM + k];
        }
      }
      // child-row tiles (an even number of rows, so pairs align): the widest
      // tile whose parent band fits 100 KB (the band as copied, its padded
      // conjugate-shifted rows, the phi-transposed rows)
      const size_t per_row = (size_t)P.nph * 32 + (size_t)(P.nph + padl + padr) * 32 + (size_t)C.nph * 32;
      auto tile_band = [&](int i0, int i1, int* lo, int* hi) {
        *lo = P.nth; *hi = 0;
        for (int i = i0; i < i1; ++i) {
          if (tq[i / 2] >= 0) {
            *lo = std::min(*lo, tq[i / 2]);
            *hi = std::max(*hi, tq[i / 2] + WTM);
          } else {
            for (int k = 0; k < TM; ++k) {
              const int tp = ttp2[(size_t)i * TM + k] & 0xffff;
              *lo = std::min(*lo, tp);
              *hi = std::max(*hi, tp + 1);
            }
          }
        }
      };
      int TI = C.nth, br = 0;
      for (;; TI = std::max(2, (TI / 2) & ~1)) {
        br = 0;
        for (int i0 = 0; i0 < C.nth; i0 += TI) {
          int lo, hi;
          tile_band(i0, std::min(C.nth, i0 + TI), &lo, &hi);
          br = std::max(br, hi - lo);
        }
        if (TI == 2 || (size_t)br * per_row <= 100 * 1024) break;
      }
      C.an2_TI = TI;
      C.an2_nit = (C.nth + TI - 1) / TI;
      C.an2_BR = br;
      C.an2_PM = PM;
      C.an2_TM = TM;
      C.an2_PADL = padl;
      C.an2_PADR = padr;
      std::vector<int> lohi2(2 * C.an2_nit);
      for (int it = 0; it < C.an2_nit; ++it)
        tile_band(it * TI, std::min(C.nth, (it + 1) * TI), &lohi2[it], &lohi2[C.an2_nit + it]);
      if ((size_t)br * per_row > 100 * 1024 || !pairs_ok) C.an2_TI = 0;   // does not fit: k_anterp1
      if ((rc = upload(c, &C.d_an2_lo, lohi2)) ||
          (rc = upload(c, &C.d_an2_ttp, ttp2)) || (rc = upload(c, &C.d_an2_tw, tw2)) ||
          (rc = upload(c, &C.d_an2_pst2, pst2)) || (rc = upload(c, &C.d_an2_pwp, pwp)) ||
          (rc = upload(c, &C.d_an2_tq, tq)) || (rc = upload(c, &C.d_an2_twq, twq)))
        return rc;
    }
    std::vector<float> ppw32(ppw.begin(), ppw.end()), tpw32(tpw.begin(), tpw.end());
    if ((rc = upload(c, &C.d_ant_pjp, ppj)) || (rc = upload(c, &C.d_ant_pw64, ppw)) ||
        (rc = upload(c, &C.d_ant_pw32, ppw32)) || (rc = upload(c, &C.d_ant_ttp, tpk)) ||
        (rc = upload(c, &C.d_ant_tw64, tpw)) || (rc = upload(c, &C.d_ant_tw32, tpw32)))
      return rc;
  }
  // shift tables exp(j k khat_p . (c_child - c_parent)), child offset (+-1/2) x child box
  std::vector<double2> sh(4 * (size_t)P.K);
  std::vector<float2> sh32(4 * (size_t)P.K);
  for (int q = 0; q < 4; ++q) {
    double dx = ((q & 1) - 0.5) * C.box, dy = ((q >> 1) - 0.5) * C.box;
    for (int k = 0; k < P.K; ++k) {
      double ph = c->k * (P.khat[3 * k] * dx + P.khat[3 * k + 1] * dy);
      sh[(size_t)q * P.K + k] = make_double2(std::cos(ph), std::sin(ph));
      sh32[(size_t)q * P.K + k] = make_float2((float)std::cos(ph), (float)std::sin(ph));
    }
  }
  std::vector<float2> sh4((size_t)4 * P.K);      // quadrant-interleaved per direction
  for (int k = 0; k < P.K; ++k)
    for (int q = 0; q < 4; ++q) sh4[(size_t)4 * k + q] = sh32[(size_t)q * P.K + k];
  if ((rc = upload(c, &C.d_shift64, sh)) || (rc = upload(c, &C.d_shift32, sh32)) ||
      (rc = upload(c, &C.d_shift4_32, sh4)))
    return rc;
  return SMR_OK;
}

int set_scene(Ctx* c, int p, const double* centres, const int* shape_ids, const int* array_ids,
              const double* eps_in, const double* mu_in, const double* eps_out, const double* mu_out) {
  if (p <= 0 || !centres || !shape_ids) return fail(c, SMR_E_INVALID_ARG, "p > 0 and host arrays required");
  if (c->shapes.empty()) return fail(c, SMR_E_SHAPE, "no shapes registered");
  if (eps_in[1] != 0 || mu_in[1] != 0 || eps_out[1] != 0 || mu_out[1] != 0 || eps_in[0] <= 0 ||
      mu_in[0] <= 0 || eps_out[0] <= 0 || mu_out[0] <= 0)
    return fail(c, SMR_E_INVALID_ARG, "only real positive permittivity/permeability are supported");
  free_scene(c);
  int npsi = c->shapes[0].n_psi();
  for (auto& s : c->shapes)
    if (s.n_psi() != npsi) return fail(c, SMR_E_SHAPE, "all shapes must share n_perp + n_par");
  c->p = p;
  c->npsi = npsi;
  c->S = (int)c->shapes.size();
  double lam = c->opts.wavelength;
  c->k = 2.0 * PI / lam * std::sqrt(eps_out[0] * mu_out[0]);
  c->zeta = std::sqrt(mu_out[0] / eps_out[0]);
  c->k_in = 2.0 * PI / lam * std::sqrt(eps_in[0] * mu_in[0]);
  c->zeta_in = std::sqrt(mu_in[0] / eps_in[0]);
  c->centres.assign(centres, centres + 3 * (size_t)p);
  c->sid.assign(shape_ids, shape_ids + p);
  for (int i = 0; i < p; ++i)
    if (c->sid[i] < 0 || c->sid[i] >= c->S) return fail(c, SMR_E_SHAPE, "shape id out of range");
  double pitch = c->opts.pitch;
  // lattice indices and finest-box offsets, per array: every array is placed
  // in its own block of a common lattice, aligned and separated so that at
  // every level up to the cap no box of one array is adjacent to, or shares a
  // parent neighbourhood with, a box of another (no near pair, no
  // interaction-list entry crosses arrays)
  std::vector<int> arr(p, 0);
  int na = 1;
  if (array_ids) {
    for (int i = 0; i < p; ++i) {
      if (array_ids[i] < 0) return fail(c, SMR_E_INVALID_ARG, "array ids must be >= 0");
      arr[i] = array_ids[i];
      na = std::max(na, arr[i] + 1);
    }
  }
  std::vector<double> ax(na, 1e300), ay(na, 1e300);
  std::vector<int> acount(na, 0);
  double zs = 0;
  for (int i = 0; i < p; ++i) {
    ax[arr[i]] = std::min(ax[arr[i]], centres[3 * i]);
    ay[arr[i]] = std::min(ay[arr[i]], centres[3 * i + 1]);
    acount[arr[i]]++;
    zs += centres[3 * i + 2];
  }
  for (int a = 0; a < na; ++a)
    if (acount[a] == 0) return fail(c, SMR_E_INVALID_ARG, "array ids must be 0..n_arrays-1 without gaps");
  c->origin[0] = ax[0];
  c->origin[1] = ay[0];
  c->z0 = zs / p;
  c->pi.resize(p);
  c->pj.resize(p);
  std::vector<int> lx(p), ly(p), ex(na, 0), ey(na, 0);
  std::vector<double> dsh(3 * (size_t)p);
  int anyd = 0;
  for (int i = 0; i < p; ++i) {
    int a = arr[i];
    double fx = (centres[3 * i] - ax[a]) / pitch, fy = (centres[3 * i + 1] - ay[a]) / pitch;
    int ix = (int)std::lround(fx), iy = (int)std::lround(fy);
    // off-lattice centres: each particle belongs to the lattice cell nearest
    // to it (its finest group) and keeps its displacement from the cell's
    // centre; within 1e-9 cells of a lattice point (rounding of the input)
    // it counts as on it
    if (std::fabs(fx - ix) <= 1e-9) fx = ix;
    if (std::fabs(fy - iy) <= 1e-9) fy = iy;
    // a centre off the mean plane z0 (a layer of a 2.5D scene) keeps its
    // height as part of the displacement; the quadtree stays in the plane
    double dz = centres[3 * i + 2] - c->z0;
    if (std::fabs(dz) <= 1e-9 * pitch) dz = 0.0;
    if (ix > (1 << 20) || iy > (1 << 20)) return fail(c, SMR_E_INVALID_ARG, "array too large");
    lx[i] = ix;
    ly[i] = iy;
    ex[a] = std::max(ex[a], ix + 1);
    ey[a] = std::max(ey[a], iy + 1);
    dsh[3 * i] = (fx - ix) * pitch;
    dsh[3 * i + 1] = (fy - iy) * pitch;
    dsh[3 * i + 2] = dz;
    if (dsh[3 * i] != 0 || dsh[3 * i + 1] != 0 || dsh[3 * i + 2] != 0) anyd = 1;
  }
  int level_cap = 1 << 20;
  std::vector<int> offx(na, 0), offy(na, 0);
  if (na > 1) {
    // each array's own top level: first s where it spans at most 2 boxes per side
    int scap = 0, emax = 0;
    for (int a = 0; a < na; ++a) {
      int sa = 0;
      while (std::max((ex[a] - 1) >> sa, (ey[a] - 1) >> sa) > 1) ++sa;
      scap = std::max(scap, sa);
      emax = std::max(emax, std::max(ex[a], ey[a]));
    }
    int M = 1 << (scap + 2);
    int stride = ((emax + 4 * (1 << scap) + M - 1) / M) * M;
    int ncol = (int)std::ceil(std::sqrt((double)na));
    for (int a = 0; a < na; ++a) { offx[a] = (a % ncol) * stride; offy[a] = (a / ncol) * stride; }
    level_cap = scap;
  }
  c->n_arrays = na;
  c->arr = arr;
  // the particles of every occupied cell, ascending; a cell holding more
  // than one makes the occupied cells the finest boxes
  std::map<std::pair<int, int>, std::vector<int>> cellp;
  int multi = 0;
  for (int i = 0; i < p; ++i) {
    c->pi[i] = lx[i] + offx[arr[i]];
    c->pj[i] = ly[i] + offy[arr[i]];
    std::vector<int>& m = cellp[std::make_pair(c->pi[i], c->pj[i])];
    m.push_back(i);
    if (m.size() > 1) multi = 1;
  }
  if (multi && !anyd) return fail(c, SMR_E_INVALID_ARG, "two particles at one centre");
  // check no particle overlaps its neighbours on the lattice (the particles
  // share one plane, so their extent across the z axis decides)
  for (auto& s : c->shapes)
    if (2 * (s.sampled ? s.lateral : s.a) >= pitch)
      return fail(c, SMR_E_INVALID_ARG, "particle width must be below the pitch");
  if (anyd) {
    // displaced particles (Sec. V, non-lattice arrays): neighbours must not
    // overlap, and every particle must lie inside the sphere of radius pitch
    // about its cell centre, so that the sources of two groups of an
    // interaction list (centres at least two cells apart) never meet and the
    // plane-wave expansion of the translation converges
    // overlap test on bounding cylinders about z: lateral radius and half
    // height of each shape
    std::vector<double> zext(c->S, 0.0);
    for (int t = 0; t < c->S; ++t) {
      const Shape& sh = c->shapes[t];
      if (!sh.sampled) zext[t] = sh.a;
      for (int q = 0; q < sh.nq; ++q) zext[t] = std::max(zext[t], std::fabs(sh.rq[4 * (size_t)q + 2]));
    }
    for (int i = 0; i < p; ++i) {
      const Shape& si = c->shapes[c->sid[i]];
      if (std::sqrt(dsh[3 * i] * dsh[3 * i] + dsh[3 * i + 1] * dsh[3 * i + 1] + dsh[3 * i + 2] * dsh[3 * i + 2]) +
              si.a >= pitch)
        return fail(c, SMR_E_INVALID_ARG, "a displaced particle reaches a pitch or more from its cell centre");
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          auto it = cellp.find({c->pi[i] + dx, c->pj[i] + dy});
          if (it == cellp.end()) continue;
          for (int j : it->second) {
            if (j == i) continue;
            const Shape& sj = c->shapes[c->sid[j]];
            const double ei = si.sampled ? si.lateral : si.a, ej = sj.sampled ? sj.lateral : sj.a;
            if (std::hypot(centres[3 * i] - centres[3 * j], centres[3 * i + 1] - centres[3 * j + 1]) <= ei + ej &&
                std::fabs(centres[3 * i + 2] - centres[3 * j + 2]) < zext[c->sid[i]] + zext[c->sid[j]])
              return fail(c, SMR_E_INVALID_ARG, "two neighbouring particles overlap");
          }
        }
    }
  }
  c->any_dshift = anyd;
  c->multi = multi;
  // ---- levels
  std::vector<int> bi(c->pi), bj(c->pj);
  std::vector<Level> levs;
  for (int s = 0;; ++s) {
    Level L;
    L.box = pitch * (double)(1 << s);
    if (s == 0 && !multi) {
      L.bi = bi;
      L.bj = bj;
    } else {
      std::vector<std::pair<int, int>> keys;
      for (size_t t = 0; t < bi.size(); ++t) keys.push_back({bj[t], bi[t]});
      std::sort(keys.begin(), keys.end());
      keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
      for (auto& kv : keys) { L.bi.push_back(kv.second); L.bj.push_back(kv.first); }
    }
    L.nbox = (int)L.bi.size();
    std::map<std::pair<int, int>, int> index;
    for (int b = 0; b < L.nbox; ++b) index[{L.bi[b], L.bj[b]}] = b;
    L.centre.resize(3 * (size_t)L.nbox);
    double half = ((double)(1 << s) - 1.0) / 2.0;
    for (int b = 0; b < L.nbox; ++b) {
      L.centre[3 * b] = c->origin[0] + ((double)L.bi[b] * (1 << s) + half) * pitch;
      L.centre[3 * b + 1] = c->origin[1] + ((double)L.bj[b] * (1 << s) + half) * pitch;
      L.centre[3 * b + 2] = c->z0;
    }
    // interaction list: parents adjacent (or equal), boxes not adjacent
    std::map<std::pair<int, int>, int> offid;
    L.il_ptr.assign(1, 0);
    for (int b = 0; b < L.nbox; ++b) {
      int ix = L.bi[b], iy = L.bj[b], px = ix >> 1, py = iy >> 1;
      for (int qx = px - 1; qx <= px + 1; ++qx)
        for (int qy = py - 1; qy <= py + 1; ++qy)
          for (int cx = 2 * qx; cx <= 2 * qx + 1; ++cx)
            for (int cy = 2 * qy; cy <= 2 * qy + 1; ++cy) {
              if (std::max(std::abs(cx - ix), std::abs(cy - iy)) <= 1) continue;
              auto it = index.find({cx, cy});
              if (it == index.end()) continue;
              std::pair<int, int> o(ix - cx, iy - cy);
              auto f = offid.find(o);
              int oid;
              if (f == offid.end()) {
                oid = (int)L.off_dx.size();
                offid[o] = oid;
                L.off_dx.push_back(o.first);
                L.off_dy.push_back(o.second);
              } else {
                oid = f->second;
              }
              L.il_src.push_back(it->second);
              L.il_off.push_back(oid);
            }
      L.il_ptr.push_back((int)L.il_src.size());
    }
    int minx = *std::min_element(L.bi.begin(), L.bi.end()), maxx = *std::max_element(L.bi.begin(), L.bi.end());
    int miny = *std::min_element(L.bj.begin(), L.bj.end()), maxy = *std::max_element(L.bj.begin(), L.bj.end());
    levs.push_back(std::move(L));
    if (std::max(maxx - minx, maxy - miny) <= 1 || s >= level_cap) break;
    for (size_t t = 0; t < bi.size(); ++t) { bi[t] >>= 1; bj[t] >>= 1; }
    if (s > 20) return fail(c, SMR_E_INVALID_ARG, "tree too deep");
  }
  while (levs.size() > 1 && levs.back().il_src.empty()) levs.pop_back();
  c->nlev = (int)levs.size();
  if (c->nlev > 16) return fail(c, SMR_E_INVALID_ARG, "more than 16 levels");
  // parents / children
  for (int s = 0; s + 1 < c->nlev; ++s) {
    Level &C = levs[s], &P = levs[s + 1];
    std::map<std::pair<int, int>, int> pidx;
    for (int b = 0; b < P.nbox; ++b) pidx[{P.bi[b], P.bj[b]}] = b;
    C.parent.resize(C.nbox);
    C.quad.resize(C.nbox);
    std::vector<std::vector<std::pair<int, int>>> ch(P.nbox);
    for (int b = 0; b < C.nbox; ++b) {
      int B = pidx[{C.bi[b] >> 1, C.bj[b] >> 1}];
      C.parent[b] = B;
      C.quad[b] = (C.bi[b] & 1) + 2 * (C.bj[b] & 1);
      ch[B].push_back({b, C.quad[b]});
    }
    P.ch_ptr.assign(1, 0);
    for (int B = 0; B < P.nbox; ++B) {
      for (auto& e : ch[B]) { P.ch_idx.push_back(e.first); P.ch_quad.push_back(e.second); }
      P.ch_ptr.push_back((int)P.ch_idx.size());
    }
  }
  c->lev = std::move(levs);
  for (int s = 0; s < c->nlev; ++s) {
    Level& L = c->lev[s];
    L.L = truncation(c, s);
    make_grid(L);
    int rc;
    if ((rc = upload(c, &L.d_khat, L.khat)) || (rc = upload(c, &L.d_w, L.w)) ||
        (rc = upload(c, &L.d_il_ptr, L.il_ptr)) || (rc = upload(c, &L.d_il_src, L.il_src)) ||
        (rc = upload(c, &L.d_il_off, L.il_off)) || (rc = upload(c, &L.d_parent, L.parent)) ||
        (rc = upload(c, &L.d_quad, L.quad)) || (rc = upload(c, &L.d_ch_ptr, L.ch_ptr)) ||
        (rc = upload(c, &L.d_ch_idx, L.ch_idx)) || (rc = upload(c, &L.d_ch_quad, L.ch_quad)))
      return rc;
  }
  for (int s = 0; s + 1 < c->nlev; ++s) {
    int rc = build_interp(c, c->lev[s], c->lev[s + 1]);
    if (rc) return rc;
  }
  // dense lattice maps and offset ids (translation tiles)
  for (int s = 0; s < c->nlev; ++s) {
    Level& L = c->lev[s];
    int x0 = *std::min_element(L.bi.begin(), L.bi.end()), x1 = *std::max_element(L.bi.begin(), L.bi.end());
    int y0 = *std::min_element(L.bj.begin(), L.bj.end()), y1 = *std::max_element(L.bj.begin(), L.bj.end());
    L.map_x0 = x0; L.map_y0 = y0; L.map_w = x1 - x0 + 1; L.map_h = y1 - y0 + 1;
    std::vector<int> bm((size_t)L.map_w * L.map_h, -1), oid(49, -1);
    for (int b = 0; b < L.nbox; ++b) bm[(size_t)(L.bj[b] - y0) * L.map_w + (L.bi[b] - x0)] = b;
    // translation tables are stored by lattice offset: row (dx + 3) * 7 + (dy + 3)
    for (size_t o = 0; o < L.off_dx.size(); ++o) {
      int g = (L.off_dx[o] + 3) * 7 + (L.off_dy[o] + 3);
      oid[g] = g;
    }
    L.ntile_x = ((x0 + L.map_w - 1) >> 2) - (x0 >> 2) + 1;
    L.ntile_y = ((y0 + L.map_h - 1) >> 2) - (y0 >> 2) + 1;
    std::vector<char> used((size_t)L.ntile_x * L.ntile_y, 0);
    for (int b = 0; b < L.nbox; ++b)
      used[(size_t)((L.bj[b] >> 2) - (y0 >> 2)) * L.ntile_x + ((L.bi[b] >> 2) - (x0 >> 2))] = 1;
    std::vector<int> tiles;
    for (size_t t = 0; t < used.size(); ++t)
      if (used[t]) tiles.push_back((int)t);
    L.ntile_ne = (int)tiles.size();
    L.ntile8_x = ((x0 + L.map_w - 1) >> 3) - (x0 >> 3) + 1;
    int nt8y = ((y0 + L.map_h - 1) >> 3) - (y0 >> 3) + 1;
    std::vector<char> used8((size_t)L.ntile8_x * nt8y, 0);
    for (int b = 0; b < L.nbox; ++b)
      used8[(size_t)((L.bj[b] >> 3) - (y0 >> 3)) * L.ntile8_x + ((L.bi[b] >> 3) - (x0 >> 3))] = 1;
    std::vector<int> tiles8;
    for (size_t t = 0; t < used8.size(); ++t)
      if (used8[t]) tiles8.push_back((int)t);
    L.ntile8_ne = (int)tiles8.size();
    // interaction list packed for the few-box kernel: source box * 64 + table row
    std::vector<int> pk(L.il_src.size());
    for (size_t e = 0; e < L.il_src.size(); ++e)
      pk[e] = L.il_src[e] * 64 + (L.off_dx[L.il_off[e]] + 3) * 7 + (L.off_dy[L.il_off[e]] + 3);
    int rc;
    if (!pk.empty() && (rc = upload(c, &L.d_il_pk, pk))) return rc;
    if ((rc = upload(c, &L.d_tiles8, tiles8))) return rc;
    if ((rc = upload(c, &L.d_boxmap, bm)) || (rc = upload(c, &L.d_offid, oid)) ||
        (rc = upload(c, &L.d_tiles, tiles)))
      return rc;
  }
  // particles grouped by shape, tiles of at most 16
  {
    std::vector<int> perm(p), tsh, tst, tcn;
    for (int i = 0; i < p; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return c->sid[a] < c->sid[b]; });
    for (int i = 0; i < p;) {
      int s = c->sid[perm[i]], j = i;
      while (j < p && c->sid[perm[j]] == s && j - i < 16) ++j;
      tsh.push_back(s); tst.push_back(i); tcn.push_back(j - i);
      i = j;
    }
    c->ntile = (int)tsh.size();
    int rc;
    if ((rc = upload(c, &c->d_perm, perm)) || (rc = upload(c, &c->d_tile_shape, tsh)) ||
        (rc = upload(c, &c->d_tile_start, tst)) || (rc = upload(c, &c->d_tile_count, tcn)))
      return rc;
  }
  // ---- near lists: self + 8 lattice neighbours; block keys (sm, sn, dx, dy)
  // on a lattice; with displaced particles every exterior block is keyed by
  // the exact centre offset as well (one block per distinct pair geometry)
  c->blk_sm.clear(); c->blk_sn.clear(); c->blk_dx.clear(); c->blk_dy.clear(); c->blk_off.clear();
  for (int s = 0; s < c->S; ++s) {
    c->blk_sm.push_back(s); c->blk_sn.push_back(s); c->blk_dx.push_back(0); c->blk_dy.push_back(0);
    c->blk_off.insert(c->blk_off.end(), {0.0, 0.0, 0.0});
  }
  std::map<std::tuple<int, int, int, int, unsigned long long, unsigned long long, unsigned long long>, int> bkey;
  auto bits = [](double v) { unsigned long long u; std::memcpy(&u, &v, sizeof u); return u; };
  c->nr_ptr.assign(1, 0);
  c->nr_col.clear();
  c->nr_blk.clear();
  for (int mu = 0; mu < p; ++mu) {
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        auto it = cellp.find({c->pi[mu] + dx, c->pj[mu] + dy});
        if (it == cellp.end()) continue;
        for (int nu : it->second) {
          int b;
          if (nu == mu) {
            b = c->sid[mu];
          } else {
            // r_mu - r_nu: the lattice offset, plus the displacements
            double ox = -dx * pitch, oy = -dy * pitch, oz = 0.0;
            if (anyd) {
              ox += dsh[3 * mu] - dsh[3 * nu];
              oy += dsh[3 * mu + 1] - dsh[3 * nu + 1];
              oz = dsh[3 * mu + 2] - dsh[3 * nu + 2];
            }
            auto key = std::make_tuple(c->sid[mu], c->sid[nu], -dx, -dy, anyd ? bits(ox) : 0ull,
                                       anyd ? bits(oy) : 0ull, anyd ? bits(oz) : 0ull);
            auto f = bkey.find(key);
            if (f == bkey.end()) {
              b = (int)c->blk_sm.size();
              bkey[key] = b;
              c->blk_sm.push_back(c->sid[mu]); c->blk_sn.push_back(c->sid[nu]);
              c->blk_dx.push_back(-dx); c->blk_dy.push_back(-dy);
              c->blk_off.insert(c->blk_off.end(), {ox, oy, oz});
            } else {
              b = f->second;
            }
          }
          c->nr_col.push_back(nu);
          c->nr_blk.push_back(b);
        }
      }
    c->nr_ptr.push_back((int)c->nr_col.size());
  }
  // the finest box of every particle, and each box's particles (CSR)
  {
    const Level& L0 = c->lev[0];
    c->cell_of.assign(p, 0);
    std::vector<int> cptr(L0.nbox + 1, 0), cidx(p);
    if (multi) {
      std::map<std::pair<int, int>, int> bidx;
      for (int b = 0; b < L0.nbox; ++b) bidx[{L0.bi[b], L0.bj[b]}] = b;
      for (int i = 0; i < p; ++i) c->cell_of[i] = bidx.at({c->pi[i], c->pj[i]});
    } else {
      for (int i = 0; i < p; ++i) c->cell_of[i] = i;
    }
    for (int i = 0; i < p; ++i) cptr[c->cell_of[i] + 1]++;
    for (int b = 0; b < L0.nbox; ++b) cptr[b + 1] += cptr[b];
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int i = 0; i < p; ++i) cidx[fill[c->cell_of[i]]++] = i;
    int rc;
    if ((rc = upload(c, &c->d_cell_of, c->cell_of)) || (rc = upload(c, &c->d_cell_ptr, cptr)) ||
        (rc = upload(c, &c->d_cell_idx, cidx)))
      return rc;
  }
  c->nblk = (int)c->blk_sm.size();
  std::vector<int> pcp(p + 1), pcc(p), pcb(p);
  for (int i = 0; i < p; ++i) { pcp[i] = i; pcc[i] = i; pcb[i] = c->sid[i]; }
  pcp[p] = p;
  std::vector<double> cen(c->centres);
  int rc;
  if ((rc = upload(c, &c->d_arr, c->arr)) || (rc = upload(c, &c->d_sid, c->sid)) || (rc = upload(c, &c->d_centres, cen)) ||
      (rc = upload(c, &c->d_dshift, dsh)) || (rc = upload(c, &c->d_nr_ptr, c->nr_ptr)) ||
      (rc = upload(c, &c->d_nr_col, c->nr_col)) || (rc = upload(c, &c->d_nr_blk, c->nr_blk)) ||
      (rc = upload(c, &c->d_pc_ptr, pcp)) || (rc = upload(c, &c->d_pc_col, pcc)) ||
      (rc = upload(c, &c->d_pc_blk, pcb)))
    return rc;
  if ((rc = build_modes(c)) || (rc = build_patterns(c)) || (rc = build_translations(c)) ||
      (rc = build_near(c)) || (rc = build_tc(c)))
    return rc;
  // the tensor-core near product groups pairs that share a block; with one
  // block per displaced pair it would run one pair per tile, so displaced
  // scenes keep the CUDA-core block-sparse product
  c->tcn_ready = false;
  if (!anyd && (rc = build_near_tc(c))) return rc;
  // device flag that the bounded waits of the staged and tensor-core kernels raise
  if (!c->d_tc_err) {
    SMR_CUDA(c, cudaMalloc((void**)&c->d_tc_err, sizeof(int)));
    SMR_CUDA(c, cudaMemset(c->d_tc_err, 0, sizeof(int)));
  }
  SMR_CUDA(c, cudaDeviceSynchronize());
  c->have_scene = true;
  return SMR_OK;
}

bool check_scene(Ctx* c) {
  if (!c->have_scene) {
    c->err = "no scene: call smr_set_scene first";
    return false;
  }
  return true;
}

long long n_unknowns(const Ctx* c) { return 2LL * c->npsi * c->p; }

int tmp_buffer(Ctx* c, size_t elems) {
  if (c->tmp_elems >= elems) return SMR_OK;
  dfree(c->d_tmp);
  SMR_CUDA(c, cudaMalloc((void**)&c->d_tmp, elems * sizeof(double2)));
  c->tmp_elems = elems;
  return SMR_OK;
}

// Column lanes of FP32 products with R > 1: R-column graph products with 1,
// 2, 4 and 8 lanes (at most R), each timed over three replays after the
// capture; the fastest is kept (a lane count must win by 2 % over a smaller
// one, so near-ties keep the smaller memory footprint).
int tune_lanes(Ctx* c, int R, cudaStream_t st) {
  const size_t n = (size_t)2 * c->npsi * c->p;
  int rc = tmp_buffer(c, 2 * n * R);
  if (rc) return rc;
  double2* X = c->d_tmp;
  double2* Y = c->d_tmp + n * R;
  SMR_CUDA(c, cudaMemsetAsync(X, 0, n * R * sizeof(double2), st));
  cudaEvent_t e0, e1;
  SMR_CUDA(c, cudaEventCreate(&e0));
  SMR_CUDA(c, cudaEventCreate(&e1));
  const int nl0 = c->n_lanes;
  int best_nl = nl0;
  float best = 1e30f;
  for (int nl = 1; nl <= 8 && nl <= R && !rc; nl *= 2) {
    c->n_lanes = nl;
    free_graphs(c);
    rc = run_matvec_graph(c, R, SMR_PREC_FP32, X, Y, st);
    float tmin = 1e30f;
    for (int k = 0; k < 3 && !rc; ++k) {
      cudaEventRecord(e0, st);
      rc = run_matvec_graph(c, R, SMR_PREC_FP32, X, Y, st);
      cudaEventRecord(e1, st);
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(c, SMR_E_CUDA, "timing a lane count");
      float ms = 0;
      if (!rc) cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
    }
    if (!rc && tmin < 0.98f * best) {
      best = tmin;
      best_nl = nl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->n_lanes = rc ? nl0 : best_nl;
  free_graphs(c);
  return rc;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

void smr_default_opts(smr_opts* o) {
  if (!o) return;
  o->device = 0;
  o->wavelength = 1.0;
  o->pitch = 0.5;
  o->L0 = 10;
  o->level_rule = SMR_LRULE_FORMULA;
  o->digits = 3.0;
  o->n_theta = 16;
  o->n_phi = 32;
}

void smr_default_solve_opts(smr_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-4;
  o->maxit = 2000;
  o->restart = 0;
  o->precond = SMR_PRECOND_BLOCKDIAG;
  o->precision = SMR_PREC_FP64;
  o->max_outer = 8;
  o->use_x0 = 0;
  o->fallback_iters = 40;
  o->near_sweeps = 1;
  o->poly_degree = 0;
}

int smr_create(smr_ctx** out, const smr_opts* opts) {
  if (!out) return SMR_E_INVALID_ARG;
  *out = nullptr;
  smr_opts o;
  smr_default_opts(&o);
  if (opts) o = *opts;
  if (o.L0 < 2 || o.pitch <= 0 || o.wavelength <= 0 || o.n_theta < 2 || o.n_phi < 4 || o.digits <= 0)
    return SMR_E_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) return SMR_E_CUDA;
  if (cudaSetDevice(o.device) != cudaSuccess) return SMR_E_CUDA;
  smr_ctx* h = new (std::nothrow) smr_ctx();
  if (!h) return SMR_E_OOM;
  h->c.opts = o;
  h->c.device = o.device;
  *out = h;
  return SMR_OK;
}

int smr_destroy(smr_ctx* h) {
  if (!h) return SMR_OK;
  cudaSetDevice(h->c.device);
  free_scene(&h->c);
  free_side(&h->c);
  nn_free(&h->c);
  if (h->c.d_tc_err) cudaFree(h->c.d_tc_err);
  if (h->c.d_red) cudaFree(h->c.d_red);
  if (h->c.h_red) cudaFreeHost(h->c.h_red);
  delete h;
  return SMR_OK;
}

const char* smr_last_error(const smr_ctx* h) { return h ? h->c.err.c_str() : "null context"; }

int smr_add_sphere(smr_ctx* h, double radius, int n_perp, int n_par, int* shape_id) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!(radius > 0) || n_perp < 0 || n_par < 0 || n_perp + n_par < 1 || n_perp + n_par > 128)
    return fail(c, SMR_E_INVALID_ARG, "radius > 0 and 1 <= n_perp + n_par <= 128 required");
  Shape sh;
  sh.a = radius;
  sh.n_perp = n_perp;
  sh.n_par = n_par;
  c->shapes.push_back(sh);
  if (shape_id) *shape_id = (int)c->shapes.size() - 1;
  return SMR_OK;
}

int smr_add_shape_sampled(smr_ctx* h, int n_q, const double* pts, const double* wts, int n_perp, int n_par,
                          const double* modes, const double* self_block, int* shape_id) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!pts || !wts || !modes || !self_block || n_q < 1 || n_q > 8192)
    return fail(c, SMR_E_INVALID_ARG, "1 <= n_q <= 8192 and non-null points, weights, modes, self block required");
  if (n_perp < 0 || n_par < 0 || n_perp + n_par < 1 || n_perp + n_par > 128)
    return fail(c, SMR_E_INVALID_ARG, "1 <= n_perp + n_par <= 128 required");
  Shape sh;
  sh.n_perp = n_perp;
  sh.n_par = n_par;
  sh.sampled = true;
  sh.nq = n_q;
  int n = n_perp + n_par;
  sh.rq.resize((size_t)n_q * 4);
  double rmax = 0;
  for (int q = 0; q < n_q; ++q) {
    double r2 = 0;
    for (int d = 0; d < 3; ++d) {
      double v = pts[3 * q + d];
      if (!std::isfinite(v)) return fail(c, SMR_E_INVALID_ARG, "non-finite quadrature point");
      sh.rq[4 * q + d] = v;
      r2 += v * v;
    }
    if (!(wts[q] >= 0) || !std::isfinite(wts[q])) return fail(c, SMR_E_INVALID_ARG, "weights must be finite and >= 0");
    sh.rq[4 * q + 3] = wts[q];
    rmax = std::max(rmax, std::sqrt(r2));
  }
  sh.a = rmax;
  for (int q = 0; q < n_q; ++q)
    sh.lateral = std::max(sh.lateral, std::hypot(sh.rq[4 * q], sh.rq[4 * q + 1]));
  sh.modes.assign(modes, modes + (size_t)n * n_q * 4);
  for (double v : sh.modes)
    if (!std::isfinite(v)) return fail(c, SMR_E_INVALID_ARG, "non-finite mode sample");
  sh.Z.resize((size_t)4 * n * n);
  for (size_t i = 0; i < sh.Z.size(); ++i) {
    sh.Z[i] = cd(self_block[2 * i], self_block[2 * i + 1]);
    if (!std::isfinite(sh.Z[i].real()) || !std::isfinite(sh.Z[i].imag()))
      return fail(c, SMR_E_INVALID_ARG, "non-finite self block");
  }
  c->shapes.push_back(std::move(sh));
  if (shape_id) *shape_id = (int)c->shapes.size() - 1;
  return SMR_OK;
}

int smr_add_shape_mesh(smr_ctx* h, int nv, const double* verts, int nt, const int* tris, int n_perp, int n_par,
                       int* shape_id) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!verts || !tris || nv < 4 || nt < 4 || nt > 1800)
    return fail(c, SMR_E_INVALID_ARG, "non-null vertices and triangles, nv >= 4, 4 <= nt <= 1800 required");
  if (n_perp < 0 || n_par < 0 || n_perp + n_par < 1 || n_perp + n_par > 128)
    return fail(c, SMR_E_INVALID_ARG, "1 <= n_perp + n_par <= 128 required");
  Shape sh;
  sh.n_perp = n_perp;
  sh.n_par = n_par;
  int rc = mesh_static_modes(c, nv, verts, nt, tris, n_perp, n_par, sh.mm);
  if (rc) return rc;
  sh.sampled = true;
  sh.mesh = true;
  sh.nq = sh.mm.nq;
  sh.rq = sh.mm.rq;
  sh.modes = sh.mm.modes;
  sh.a = 0;
  for (int v = 0; v < nv; ++v) {
    const double* x = verts + 3 * v;
    sh.a = std::max(sh.a, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
    sh.lateral = std::max(sh.lateral, std::hypot(x[0], x[1]));
  }
  c->shapes.push_back(std::move(sh));
  if (shape_id) *shape_id = (int)c->shapes.size() - 1;
  return SMR_OK;
}

int smr_add_shape_rotated(smr_ctx* h, int base, double angle, int* shape_id) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (base < 0 || base >= (int)c->shapes.size()) return fail(c, SMR_E_SHAPE, "base shape id out of range");
  if (!std::isfinite(angle)) return fail(c, SMR_E_INVALID_ARG, "angle must be finite");
  if (!c->shapes[base].sampled)
    return fail(c, SMR_E_SHAPE, "closed-form spheres are unchanged by rotation: add the sphere again");
  // the rotated particle's modes are the base modes carried by the rotation
  // R about z: psi'(R r) = R psi(r); the surface divergence and the weights
  // are unchanged, and so is the self block
  Shape sh = c->shapes[base];
  const double cs = std::cos(angle), sn = std::sin(angle);
  auto rot = [&](double* v) {
    const double x = v[0], y = v[1];
    v[0] = cs * x - sn * y;
    v[1] = sn * x + cs * y;
  };
  for (int q = 0; q < sh.nq; ++q) rot(&sh.rq[4 * (size_t)q]);
  for (size_t i = 0; i < sh.modes.size(); i += 4) rot(&sh.modes[i]);
  // a meshed base keeps its mesh data (sh.mm: RWG coefficients, eigenvalues
  // and the geometry that assembles self blocks) unrotated: the coefficients
  // and eigenvalues are the same, and the self block is taken from the base
  sh.rot_base = c->shapes[base].rot_base >= 0 ? c->shapes[base].rot_base : base;
  sh.rot_angle = c->shapes[base].rot_angle + angle;
  c->shapes.push_back(std::move(sh));
  if (shape_id) *shape_id = (int)c->shapes.size() - 1;
  return SMR_OK;
}

int smr_shape_modes(smr_ctx* h, int shape_id, int* n_psi, int* n_edges, double* M, double* gamma) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (shape_id < 0 || shape_id >= (int)c->shapes.size() || !c->shapes[shape_id].mesh)
    return fail(c, SMR_E_INVALID_ARG, "not the id of a meshed shape");
  const Shape& sh = c->shapes[shape_id];
  if (n_psi) *n_psi = sh.n_psi();
  if (n_edges) *n_edges = sh.mm.ne;
  if (M) std::copy(sh.mm.M.begin(), sh.mm.M.end(), M);
  if (gamma) std::copy(sh.mm.gamma.begin(), sh.mm.gamma.end(), gamma);
  return SMR_OK;
}

int smr_self_block(smr_ctx* h, int shape_id, double* Z) {
  if (!h || !Z) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (shape_id < 0 || shape_id >= (int)c->shapes.size()) return fail(c, SMR_E_INVALID_ARG, "shape id out of range");
  const std::vector<cd>& z = c->shapes[shape_id].Z;
  for (size_t i = 0; i < z.size(); ++i) {
    Z[2 * i] = z[i].real();
    Z[2 * i + 1] = z[i].imag();
  }
  return SMR_OK;
}

int smr_mesh_static_modes(int nv, const double* verts, int nt, const int* tris, int n_perp, int n_par,
                          int* n_edges, double* M, double* gamma) {
  if (!verts || !tris || nv < 4 || nt < 4 || nt > 1800 || n_perp < 0 || n_par < 0 || n_perp + n_par < 1)
    return SMR_E_INVALID_ARG;
  Ctx tmp;
  MeshModes mm;
  int rc = mesh_static_modes(&tmp, nv, verts, nt, tris, n_perp, n_par, mm);
  if (rc) return rc;
  if (n_edges) *n_edges = mm.ne;
  if (M) std::copy(mm.M.begin(), mm.M.end(), M);
  if (gamma) std::copy(mm.gamma.begin(), mm.gamma.end(), gamma);
  return SMR_OK;
}

int smr_set_scene(smr_ctx* h, int p, const double* centres, const int* shape_ids, const double eps_in[2],
                  const double mu_in[2], const double eps_out[2], const double mu_out[2]) {
  if (!h || !eps_in || !mu_in || !eps_out || !mu_out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, SMR_E_CUDA, "cudaSetDevice");
  int rc = set_scene(c, p, centres, shape_ids, nullptr, eps_in, mu_in, eps_out, mu_out);
  if (rc) {
    std::string msg = c->err;
    free_scene(c);
    c->err = msg;
  }
  return rc;
}

int smr_set_scene_arrays(smr_ctx* h, int p, const double* centres, const int* shape_ids,
                         const int* array_ids, const double eps_in[2], const double mu_in[2],
                         const double eps_out[2], const double mu_out[2]) {
  if (!h || !eps_in || !mu_in || !eps_out || !mu_out || !array_ids) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, SMR_E_CUDA, "cudaSetDevice");
  int rc = set_scene(c, p, centres, shape_ids, array_ids, eps_in, mu_in, eps_out, mu_out);
  if (rc) {
    std::string msg = c->err;
    free_scene(c);
    c->err = msg;
  }
  return rc;
}

int smr_info(smr_ctx* h, smr_info_t* info) {
  if (!h || !info) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  std::memset(info, 0, sizeof(*info));
  info->p = c->p;
  info->n_psi = c->npsi;
  info->n_shapes = c->S;
  info->n_levels = c->nlev;
  info->n_arrays = c->n_arrays;
  info->n_unknowns = n_unknowns(c);
  double bytes = 0;
  for (int s = 0; s < c->nlev; ++s) {
    const Level& L = c->lev[s];
    info->L[s] = L.L;
    info->K[s] = L.K;
    info->n_box[s] = L.nbox;
    info->n_il[s] = (int)L.il_src.size();
    bytes += 2.0 * L.nbox * L.K * 4 * 16 + (double)L.off_dx.size() * L.K * 24;
  }
  info->n_near_pairs = (long long)c->nr_col.size();
  info->n_near_blocks = c->nblk;
  bytes += (double)c->nblk * 4 * c->npsi * c->npsi * 24;
  info->device_bytes = bytes;
  info->column_lanes = c->n_lanes;
  return SMR_OK;
}

int smr_rhs_plane_waves(smr_ctx* h, int R, const double* khat, const double* pol, void* b, void* stream) {
  if (!h || R <= 0 || !khat || !pol || !b) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> kh(khat, khat + 3 * (size_t)R);
  std::vector<double2> pl(3 * (size_t)R);
  for (int i = 0; i < 3 * R; ++i) pl[i] = make_double2(pol[2 * i], pol[2 * i + 1]);
  double* d_k = nullptr;
  double2* d_p = nullptr;
  int rc;
  if ((rc = upload(c, &d_k, kh)) || (rc = upload(c, &d_p, pl))) return rc;
  rc = launch_rhs(c, R, d_k, d_p, (double2*)b, st);
  cudaStreamSynchronize(st);
  cudaFree(d_k);
  cudaFree(d_p);
  return rc;
}

int smr_matvec(smr_ctx* h, int R, const void* x, void* y, int precision, void* stream) {
  if (!h || R <= 0 || R > 256 || !x || !y) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (precision != SMR_PREC_FP64 && precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  cudaStream_t st = (cudaStream_t)stream;
  return run_product(c, R, precision, (const double2*)x, (double2*)y, st);
}

int smr_matvec_graph(smr_ctx* h, int R, const void* x, void* y, int precision, void* stream) {
  if (!h || R <= 0 || R > 256 || !x || !y) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (precision != SMR_PREC_FP64 && precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  return run_matvec_graph(c, R, precision, (const double2*)x, (double2*)y, (cudaStream_t)stream);
}

int smr_matvec_parts(smr_ctx* h, int R, const void* x, void* y_near, void* y_far, int precision,
                     void* stream) {
  if (!h || R <= 0 || R > 256 || !x) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (precision != SMR_PREC_FP64 && precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = prep_x32(c, R, precision, (const double2*)x, st);
  if (!rc && y_near) rc = run_near(c, R, precision, (const double2*)x, (double2*)y_near, st);
  if (!rc && y_far) rc = run_far(c, R, precision, (const double2*)x, (double2*)y_far, false, st);
  c->x32_of = nullptr;
  return rc;
}

int smr_matvec_host(smr_ctx* h, int R, const double* x, double* y, int precision, void* stream) {
  if (!h || R <= 0 || R > 256 || !x || !y) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  size_t n = (size_t)n_unknowns(c) * R;
  int rc = tmp_buffer(c, 2 * n);
  if (rc) return rc;
  double2* dx = c->d_tmp;
  double2* dy = c->d_tmp + n;
  SMR_CUDA(c, cudaMemcpyAsync(dx, x, n * sizeof(double2), cudaMemcpyHostToDevice, st));
  rc = smr_matvec(h, R, dx, dy, precision, stream);
  if (rc) return rc;
  SMR_CUDA(c, cudaMemcpyAsync(y, dy, n * sizeof(double2), cudaMemcpyDeviceToHost, st));
  SMR_CUDA(c, cudaStreamSynchronize(st));
  return tc_check(c);
}

int smr_precond(smr_ctx* h, int R, const void* r, void* z, int precision, void* stream) {
  if (!h || R <= 0 || R > 256 || !r || !z) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  return run_precond(c, R, precision, (const double2*)r, (double2*)z, (cudaStream_t)stream);
}

int smr_solve(smr_ctx* h, int R, const void* b, void* x, const smr_solve_opts* opts, smr_solve_stats* stats,
              void* stream) {
  if (!h || R <= 0 || R > 256 || !b || !x) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  smr_solve_opts o;
  smr_default_solve_opts(&o);
  if (opts) o = *opts;
  if (o.precision != SMR_PREC_FP64 && o.precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  if (o.precond != SMR_PRECOND_NONE && o.precond != SMR_PRECOND_BLOCKDIAG && o.precond != SMR_PRECOND_LEARNED &&
      o.precond != SMR_PRECOND_NEAR && o.precond != SMR_PRECOND_CLUSTER)
    return fail(c, SMR_E_INVALID_ARG, "unknown preconditioner");
  if (o.precond == SMR_PRECOND_CLUSTER) {
    int rb = build_clusters(c);
    if (rb) return rb;
  }
  if (o.precond == SMR_PRECOND_NEAR && (o.near_sweeps < 1 || o.near_sweeps > 8))
    return fail(c, SMR_E_INVALID_ARG, "near_sweeps must be in 1..8");
  if (o.poly_degree < 0 || o.poly_degree == 1 || o.poly_degree > 16)
    return fail(c, SMR_E_INVALID_ARG, "poly_degree must be 0 (off) or in 2..16");
  if (o.precond == SMR_PRECOND_LEARNED && (R != 1 || !c->lpc_ready))
    return fail(c, SMR_E_STATE, "SMR_PRECOND_LEARNED needs R = 1 and smr_nn_precond first");
  int rc = solve(c, R, (const double2*)b, (double2*)x, &o, stats, (cudaStream_t)stream);
  int rt = tc_check(c);
  return rc ? rc : rt;
}

int smr_precond_cluster(smr_ctx* h, int R, const void* r, void* z, int precision, void* stream) {
  if (!h || R <= 0 || R > 256 || !r || !z) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (precision != SMR_PREC_FP64 && precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  int rc = build_clusters(c);
  if (rc) return rc;
  return run_cluster(c, R, precision, (const double2*)r, (double2*)z, (cudaStream_t)stream);
}

int smr_set_tensor_cores(smr_ctx* h, int enable) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  cudaSetDevice(c->device);
  c->tc_enable = enable != 0;
  free_graphs(c);                              // captured products used the old setting
  return SMR_OK;
}

int smr_set_variant(smr_ctx* h, int step, int level, int precision, int variant) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (precision != SMR_PREC_FP64 && precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  if (level < -1 || level >= c->nlev) return fail(c, SMR_E_INVALID_ARG, "level out of range");
  const int q = precision == SMR_PREC_FP64 ? 0 : 1;
  const bool ok = (step == SMR_STEP_TRANSLATE && variant >= 0 && variant <= 5) ||
                  (step == SMR_STEP_INTERPOLATE && variant >= 0 && variant <= 3) ||
                  (step == SMR_STEP_ANTERPOLATE && (variant >= 0 && variant <= 2 || variant == 4 || variant == 5));
  if (!ok) return fail(c, SMR_E_INVALID_ARG, "unknown step or variant");
  for (int s = (level < 0 ? 0 : level); s < (level < 0 ? c->nlev : level + 1); ++s) {
    Level& L = c->lev[s];
    if (step == SMR_STEP_TRANSLATE) L.tune_tr[q] = variant;
    else if (step == SMR_STEP_INTERPOLATE) L.tune_ip[q] = variant;
    else L.tune_an[q] = variant;
  }
  free_graphs(c);                              // captured products used the old variants
  return SMR_OK;
}

int smr_set_wait_limit(smr_ctx* h, long long rounds) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (rounds > 0x7fffffffLL) return fail(c, SMR_E_INVALID_ARG, "wait limit above 2^31 - 1 rounds");
  c->tc_spin = rounds < 0 ? (1u << 24) : (uint32_t)rounds;
  free_graphs(c);                              // captured products carry the old limit
  return SMR_OK;
}

int smr_set_column_lanes(smr_ctx* h, int lanes) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (lanes < 1 || lanes > 16) return fail(c, SMR_E_INVALID_ARG, "lanes must be in 1..16");
  cudaSetDevice(c->device);
  c->n_lanes = lanes;
  free_graphs(c);                              // captured products hold the old lane count
  return SMR_OK;
}

int smr_set_overlap(smr_ctx* h, int enable) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  cudaSetDevice(c->device);
  c->overlap = enable != 0;
  free_graphs(c);                              // captured products hold the old launch order
  return SMR_OK;
}

int smr_sync(smr_ctx* h, void* stream) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  cudaSetDevice(c->device);
  SMR_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
  return tc_check(c);
}

int smr_far_field(smr_ctx* h, int R, const void* x, int n_dir, const double* dirs, void* F, void* stream) {
  if (!h || R <= 0 || !x || n_dir <= 0 || !dirs || !F) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  std::vector<double> d(dirs, dirs + 3 * (size_t)n_dir);
  double* dd = nullptr;
  int rc = upload(c, &dd, d);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = launch_far_field(c, R, (const double2*)x, n_dir, dd, (double2*)F, st);
  cudaStreamSynchronize(st);
  cudaFree(dd);
  return rc;
}

int smr_cross_sections(smr_ctx* h, int R, const void* x, int n_theta, const double* khat,
                       const double* pol, double* csca, double* cext, void* stream) {
  if (!h || R <= 0 || !x || n_theta < 1 || n_theta > 2048 || !khat || !pol || !csca || !cext)
    return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  cudaSetDevice(c->device);
  // Gauss-Legendre in cos(theta) times the trapezoid rule in phi: exact for
  // band-limited |F|^2 up to degree 2 n_theta - 1 in each.
  std::vector<double> xg, wg;
  hm::gauss_legendre(n_theta, xg, wg);
  int n_phi = 2 * n_theta, n_sca = n_theta * n_phi;
  std::vector<double> dirs(3 * ((size_t)n_sca + R)), W(n_sca);
  for (int i = 0; i < n_theta; ++i) {
    double st = std::sqrt(std::max(0.0, 1.0 - xg[i] * xg[i]));
    for (int j = 0; j < n_phi; ++j) {
      double ph = 2.0 * M_PI * j / n_phi;
      size_t d = (size_t)i * n_phi + j;
      dirs[3 * d] = st * std::cos(ph);
      dirs[3 * d + 1] = st * std::sin(ph);
      dirs[3 * d + 2] = xg[i];
      W[d] = wg[i] * 2.0 * M_PI / n_phi;
    }
  }
  std::vector<double2> pl(3 * (size_t)R);
  for (int r = 0; r < R; ++r) {
    const double* kr = khat + 3 * (size_t)r;
    double nk = std::sqrt(kr[0] * kr[0] + kr[1] * kr[1] + kr[2] * kr[2]);
    double np = 0;
    for (int i = 0; i < 3; ++i) {
      pl[3 * r + i] = make_double2(pol[6 * r + 2 * i], pol[6 * r + 2 * i + 1]);
      np += pol[6 * r + 2 * i] * pol[6 * r + 2 * i] + pol[6 * r + 2 * i + 1] * pol[6 * r + 2 * i + 1];
    }
    if (!(nk > 0) || !(np > 0))
      return fail(c, SMR_E_INVALID_ARG, "khat and pol must be non-zero for every column");
    for (int i = 0; i < 3; ++i) dirs[3 * ((size_t)n_sca + r) + i] = kr[i] / nk;
  }
  double *d_dirs = nullptr, *d_w = nullptr, *d_cs = nullptr;
  double2* d_pol = nullptr;
  int rc;
  if ((rc = upload(c, &d_dirs, dirs)) || (rc = upload(c, &d_w, W)) || (rc = upload(c, &d_pol, pl))) {
    cudaFree(d_dirs);
    cudaFree(d_w);
    return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> cs(2 * (size_t)R);
  if (cudaMalloc((void**)&d_cs, cs.size() * sizeof(double)) != cudaSuccess) {
    rc = fail(c, SMR_E_OOM, "cross sections: out of device memory");
  } else {
    rc = launch_cross_sections(c, R, (const double2*)x, n_sca, d_dirs, d_w, d_pol, d_cs, st);
    cudaStreamSynchronize(st);
    if (rc == SMR_OK &&
        cudaMemcpy(cs.data(), d_cs, cs.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = fail(c, SMR_E_CUDA, "cross sections: copy back failed");
  }
  cudaFree(d_dirs);
  cudaFree(d_w);
  cudaFree(d_pol);
  cudaFree(d_cs);
  if (rc == SMR_OK)
    for (int r = 0; r < R; ++r) {
      csca[r] = cs[2 * r];
      cext[r] = cs[2 * r + 1];
    }
  return rc;
}

int smr_near_field(smr_ctx* h, int R, const void* x, int n_pt, const double* pts, void* EH, void* stream) {
  if (!h || R <= 0 || !x || n_pt <= 0 || !pts || !EH) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  std::vector<double> d(pts, pts + 3 * (size_t)n_pt);
  double* dd = nullptr;
  int rc = upload(c, &dd, d);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = launch_near_field(c, R, (const double2*)x, n_pt, dd, (double2*)EH, st);
  cudaStreamSynchronize(st);
  cudaFree(dd);
  return rc;
}

int smr_profile_matvec(smr_ctx* h, int R, const void* x, void* y, int precision, smr_launch_t* out,
                       int n_max, int* n_out, void* stream) {
  if (!h || R <= 0 || R > 256 || !x || !y || (n_max > 0 && !out)) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  std::vector<ProfRec> recs;
  c->prof = &recs;
  int rc = smr_matvec(h, R, x, y, precision, stream);
  c->prof = nullptr;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  for (size_t i = 0; i < recs.size(); ++i) {
    float ms = 0.f;
    if (rc == SMR_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, recs[i].a, recs[i].b);
    if ((int)i < n_max) {
      std::memset(&out[i], 0, sizeof(smr_launch_t));
      std::strncpy(out[i].name, recs[i].name, sizeof(out[i].name) - 1);
      out[i].level = recs[i].level;
      out[i].bytes = recs[i].bytes;
      out[i].flops = recs[i].flops;
      out[i].ms = ms;
    }
    cudaEventDestroy(recs[i].a);
    cudaEventDestroy(recs[i].b);
  }
  if (n_out) *n_out = (int)recs.size();
  if (rc) return rc;
  if (e != cudaSuccess) return fail(c, SMR_E_CUDA, cudaGetErrorString(e));
  return SMR_OK;
}

// ---------------------------------------------------------------- autotuning of launch variants
namespace {
// per (kernel name, level) the fastest of `reps` profiled products
int profile_min(smr_ctx* h, int R, const void* x, void* y, int prec, int reps, void* stream,
                std::map<std::pair<std::string, int>, double>& best) {
  Ctx* c = &h->c;
  best.clear();
  for (int r = 0; r < reps; ++r) {
    std::vector<ProfRec> recs;
    c->prof = &recs;
    int rc = smr_matvec(h, R, x, y, prec, stream);
    c->prof = nullptr;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    // a step may take several launches (the near product runs one per
    // lattice offset): sum them per product, keep the fastest product
    std::map<std::pair<std::string, int>, double> sum;
    for (auto& q : recs) {
      float ms = 0.f;
      if (rc == SMR_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, q.a, q.b);
      sum[std::make_pair(std::string(q.name), q.level)] += ms;
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
    for (auto& kv : sum) {
      auto it = best.find(kv.first);
      if (it == best.end() || kv.second < it->second) best[kv.first] = kv.second;
    }
    if (rc) return rc;
    if (e != cudaSuccess) return fail(c, SMR_E_CUDA, cudaGetErrorString(e));
  }
  return SMR_OK;
}
}  // namespace

int smr_autotune(smr_ctx* h, int R, int precision, void* stream) {
  // the variants are timed on single-column products; FP32 products with
  // R > 1 run their columns through the same single-column kernels
  if (!h || R < 1 || R > 256) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (precision != SMR_PREC_FP64 && precision != SMR_PREC_FP32)
    return fail(c, SMR_E_INVALID_ARG, "precision must be SMR_PREC_FP64 or SMR_PREC_FP32");
  const int q = precision == SMR_PREC_FP64 ? 0 : 1;
  size_t n = (size_t)n_unknowns(c);
  int rc = tmp_buffer(c, 2 * n);
  if (rc) return rc;
  double2* x = c->d_tmp;
  double2* y = c->d_tmp + n;
  SMR_CUDA(c, cudaMemsetAsync(x, 0, n * sizeof(double2), (cudaStream_t)stream));
  std::map<std::pair<std::string, int>, double> t;
  // translation: 8x8 tiles (full, half direction chunk) and 4x4 tiles
  std::vector<std::vector<double>> ttr(c->nlev, std::vector<double>(6, 1e30));
  std::vector<std::vector<double>> tip(c->nlev, std::vector<double>(4, 1e30));
  std::vector<std::vector<double>> tan_(c->nlev, std::vector<double>(6, 1e30));
  const int anv[6] = {0, 0, 1, 2, 4, 5};       // anterpolation variant timed in trial v
  double agg[2] = {1e30, 1e30}, rec[2] = {1e30, 1e30}, nea[2] = {1e30, 1e30};
  const int agg0 = c->tune_tc_agg, rec0 = c->tune_tc_rec, nea0 = c->tune_tc_near;
  // trial 5 times the per-parent FP32 anterpolation and the whole-level
  // translation (levels of at most 256 boxes), the rest at their first variants
  for (int v = 1; v <= 5; ++v) {
    // variant 4 (few-box kernel) only where a level has at most 1024 boxes
    for (auto& L : c->lev) {
      L.tune_tr[q] = (v == 4 && L.nbox > 1024) || (v == 5 && L.nbox > 256) ? 1 : v;
      // interpolation: the built-in rule (staged kernel in FP32), k_interp1
      // with the full or the half theta-row tile
      L.tune_ip[q] = (v == 2) ? 2 : (v == 3 ? 1 : (v == 5 && q == 1 ? 3 : 0));
      L.tune_an[q] = anv[v];
    }
    c->tune_tc_agg = c->tune_tc_rec = c->tune_tc_near = (v == 3) ? 0 : 1;
    if ((rc = profile_min(h, 1, x, y, precision, 3, stream, t))) break;
    for (int s = 0; s < c->nlev; ++s) {
      auto it = t.find({"translate", s});
      if (it != t.end() && c->lev[s].tune_tr[q] == v) ttr[s][v] = it->second;
      auto an = t.find({"anterpolate", s});
      if (an != t.end()) tan_[s][anv[v]] = std::min(tan_[s][anv[v]], an->second);
      auto ip = t.find({"interpolate", s});
      const int iv = c->lev[s].tune_ip[q];
      if (ip != t.end()) tip[s][iv] = std::min(tip[s][iv], ip->second);
    }
    int tc = (v == 3) ? 0 : 1;
    auto a = t.find({"aggregate", 0});
    if (a != t.end()) agg[tc] = std::min(agg[tc], a->second);
    auto r = t.find({"receive", 0});
    if (r != t.end()) rec[tc] = std::min(rec[tc], r->second);
    auto nr = t.find({"near", -1});
    if (nr != t.end()) nea[tc] = std::min(nea[tc], nr->second);
  }
  for (int s = 0; s < c->nlev; ++s) {
    Level& L = c->lev[s];
    int bv = 1;
    for (int v = 2; v <= 5; ++v)
      if (ttr[s][v] < ttr[s][bv]) bv = v;
    L.tune_tr[q] = rc ? 0 : bv;
    int bi = 0;
    for (int v = 1; v <= 3; ++v)
      if (tip[s][v] < tip[s][bi]) bi = v;
    L.tune_ip[q] = rc ? 0 : bi;
    int ba = 0;
    for (int v = 1; v <= 5; ++v)
      if (tan_[s][v] < tan_[s][ba]) ba = v;
    L.tune_an[q] = rc ? 0 : ba;
  }
  c->tune_tc_agg = agg0;
  c->tune_tc_rec = rec0;
  c->tune_tc_near = nea0;
  if (q == 1) {                                // the tensor-core steps exist in FP32 only
    c->tune_tc_agg = rc ? -1 : (agg[1] <= agg[0] ? 1 : 0);
    c->tune_tc_rec = rc ? -1 : (rec[1] <= rec[0] ? 1 : 0);
    // the near product on the tensor cores only when clearly faster: the two
    // paths are close on single right-hand sides, and a stable choice keeps
    // the launch sequence the same from one tuning to the next
    c->tune_tc_near = rc ? -1 : (nea[1] < 0.95 * nea[0] ? 1 : 0);
  }
  free_graphs(c);                              // captured products used the trial variants
  if (!rc && q == 1 && R > 1 && c->split_cols) rc = tune_lanes(c, R, (cudaStream_t)stream);
  return rc;
}

// ---------------------------------------------------------------- per-array incidence and the learned guess
namespace {
int upload_inc(Ctx* c, int n, const double* khat, const double* pol, double** dk, double** dp) {
  std::vector<double> kh(khat, khat + 3 * (size_t)n), pl(pol, pol + 6 * (size_t)n);
  int rc = upload(c, dk, kh);
  if (rc) return rc;
  return upload(c, dp, pl);
}
}  // namespace

int smr_rhs_plane_waves_arrays(smr_ctx* h, const double* khat, const double* pol, void* b, void* stream) {
  if (!h || !khat || !pol || !b) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  double *dk = nullptr, *dp = nullptr;
  int rc = upload_inc(c, c->n_arrays, khat, pol, &dk, &dp);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = launch_rhs_arrays(c, dk, (const double2*)dp, (double2*)b, st);
  cudaStreamSynchronize(st);
  cudaFree(dk);
  cudaFree(dp);
  return rc;
}

int smr_nn_init(smr_ctx* h, int width, unsigned long long seed) {
  if (!h) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  return nn_init(c, width, seed);
}

long long smr_nn_num_params(smr_ctx* h) { return h ? h->c.nn.np : 0; }

int smr_nn_get_params(smr_ctx* h, float* out, long long n) {
  if (!h || !out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!c->nn.p32 || n != c->nn.np) return fail(c, SMR_E_INVALID_ARG, "parameter count mismatch");
  SMR_CUDA(c, cudaMemcpy(out, c->nn.p32, n * sizeof(float), cudaMemcpyDeviceToHost));
  return SMR_OK;
}

int smr_nn_set_params(smr_ctx* h, const float* in, long long n) {
  if (!h || !in) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!c->nn.p32 || n != c->nn.np) return fail(c, SMR_E_INVALID_ARG, "parameter count mismatch");
  SMR_CUDA(c, cudaMemcpy(c->nn.p32, in, n * sizeof(float), cudaMemcpyHostToDevice));
  std::vector<float> z((size_t)n, 0.f);
  SMR_CUDA(c, cudaMemcpy(c->nn.m, z.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  SMR_CUDA(c, cudaMemcpy(c->nn.v, z.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  c->nn.step = 0;
  // refresh the BF16 copies through one zero-learning-rate Adam step
  SMR_CUDA(c, cudaMemset(c->nn.g, 0, n * sizeof(float)));
  int rc = nn_adam(c, 0.f, 0);
  c->nn.step = 0;
  if (rc) return rc;
  SMR_CUDA(c, cudaDeviceSynchronize());
  return SMR_OK;
}

int smr_nn_features(smr_ctx* h, const double* khat, const double* pol, float* feat, void* stream) {
  if (!h || !khat || !pol || !feat) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  double *dk = nullptr, *dp = nullptr;
  int rc = upload_inc(c, c->n_arrays, khat, pol, &dk, &dp);
  if (rc) return rc;
  rc = nn_features(c, dk, dp, feat, (cudaStream_t)stream);
  cudaFree(dk);
  cudaFree(dp);
  return rc;
}

int smr_nn_targets(smr_ctx* h, const double* khat, const void* x, double scale, float* tgt, void* stream) {
  if (!h || !khat || !x || !tgt || !(scale > 0)) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  std::vector<double> kh(khat, khat + 3 * (size_t)c->n_arrays);
  double* dk = nullptr;
  int rc = upload(c, &dk, kh);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = nn_targets(c, dk, (const double2*)x, scale, tgt, st);
  cudaStreamSynchronize(st);
  cudaFree(dk);
  return rc;
}

int smr_nn_train_step(smr_ctx* h, int n, const float* feat, const int* idx, const float* tgt, float lr,
                      double* loss, void* stream) {
  if (!h || !feat || !tgt || n <= 0) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = nn_forward_backward(c, n, feat, idx, tgt, true, loss, st);
  if (rc) return rc;
  return nn_adam(c, lr, st);
}

int smr_nn_loss_grad(smr_ctx* h, int n, const float* feat, const int* idx, const float* tgt, double* loss,
                     float* grad, void* stream) {
  if (!h || !feat || !tgt || n <= 0) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = nn_forward_backward(c, n, feat, idx, tgt, true, loss, st);
  if (rc) return rc;
  if (grad) {
    SMR_CUDA(c, cudaMemcpyAsync(grad, c->nn.g, c->nn.np * sizeof(float), cudaMemcpyDeviceToHost, st));
    SMR_CUDA(c, cudaStreamSynchronize(st));
  }
  return SMR_OK;
}

int smr_nn_predict(smr_ctx* h, const double* khat, const double* pol, double scale, void* x0, void* stream) {
  if (!h || !khat || !pol || !x0 || !(scale > 0)) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (!c->nn.p32) return fail(c, SMR_E_STATE, "call smr_nn_init first");
  double *dk = nullptr, *dp = nullptr;
  int rc = upload_inc(c, c->n_arrays, khat, pol, &dk, &dp);
  if (rc) return rc;
  rc = nn_predict(c, dk, dp, scale, (double2*)x0, (cudaStream_t)stream);
  cudaFree(dk);
  cudaFree(dp);
  return rc;
}

int smr_nn_precond(smr_ctx* h, const double* khat, const double* pol, double scale, const void* b, void* stream) {
  if (!h || !khat || !pol || !b || !(scale > 0)) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (!c->nn.p32) return fail(c, SMR_E_STATE, "call smr_nn_init first");
  double *dk = nullptr, *dp = nullptr;
  int rc = upload_inc(c, c->n_arrays, khat, pol, &dk, &dp);
  if (rc) return rc;
  rc = nn_precond(c, dk, dp, scale, (const double2*)b, (cudaStream_t)stream);
  cudaFree(dk);
  cudaFree(dp);
  return rc;
}

int smr_copy_pattern(smr_ctx* h, int shape, double* out) {
  if (!h || !out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (shape < 0 || shape >= c->S) return fail(c, SMR_E_SHAPE, "shape id out of range");
  size_t n = (size_t)c->npsi * 2 * c->lev[0].K;
  SMR_CUDA(c, cudaMemcpy(out, c->d_P64 + (size_t)shape * n, n * sizeof(double2), cudaMemcpyDeviceToHost));
  return SMR_OK;
}

int smr_copy_translation(smr_ctx* h, int level, int dx, int dy, double* out) {
  if (!h || !out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (level < 0 || level >= c->nlev) return fail(c, SMR_E_INVALID_ARG, "level out of range");
  Level& L = c->lev[level];
  for (size_t o = 0; o < L.off_dx.size(); ++o)
    if (L.off_dx[o] == dx && L.off_dy[o] == dy) {
      size_t row = (size_t)(dx + 3) * 7 + (dy + 3);
      SMR_CUDA(c, cudaMemcpy(out, L.d_T64 + row * L.K, L.K * sizeof(double2), cudaMemcpyDeviceToHost));
      return SMR_OK;
    }
  return fail(c, SMR_E_INVALID_ARG, "offset not in this level's interaction lists");
}

int smr_copy_near_block(smr_ctx* h, int sm, int sn, int dx, int dy, double* out) {
  if (!h || !out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  int n2 = 2 * c->npsi;
  for (int b = 0; b < c->nblk; ++b)
    if (c->blk_sm[b] == sm && c->blk_sn[b] == sn && c->blk_dx[b] == dx && c->blk_dy[b] == dy) {
      std::vector<double2> t((size_t)n2 * n2);
      SMR_CUDA(c, cudaMemcpy(t.data(), c->d_B64 + (size_t)b * n2 * n2, t.size() * sizeof(double2),
                             cudaMemcpyDeviceToHost));
      for (int i = 0; i < n2; ++i)
        for (int j = 0; j < n2; ++j) {
          out[2 * ((size_t)i * n2 + j)] = t[(size_t)j * n2 + i].x;
          out[2 * ((size_t)i * n2 + j) + 1] = t[(size_t)j * n2 + i].y;
        }
      return SMR_OK;
    }
  return fail(c, SMR_E_INVALID_ARG, "no such near block in this scene");
}

int smr_copy_pair_block(smr_ctx* h, int mu, int nu, double* out) {
  if (!h || !out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (mu < 0 || mu >= c->p || nu < 0 || nu >= c->p) return fail(c, SMR_E_INVALID_ARG, "particle index out of range");
  const int n2 = 2 * c->npsi;
  for (int e = c->nr_ptr[mu]; e < c->nr_ptr[mu + 1]; ++e) {
    if (c->nr_col[e] != nu) continue;
    std::vector<double2> t((size_t)n2 * n2);
    SMR_CUDA(c, cudaMemcpy(t.data(), c->d_B64 + (size_t)c->nr_blk[e] * n2 * n2, t.size() * sizeof(double2),
                           cudaMemcpyDeviceToHost));
    for (int i = 0; i < n2; ++i)
      for (int j = 0; j < n2; ++j) {
        out[2 * ((size_t)i * n2 + j)] = t[(size_t)j * n2 + i].x;
        out[2 * ((size_t)i * n2 + j) + 1] = t[(size_t)j * n2 + i].y;
      }
    return SMR_OK;
  }
  return fail(c, SMR_E_INVALID_ARG, "the two particles are not a near pair");
}

int smr_copy_level(smr_ctx* h, int level, int kind, double* out, size_t n_doubles) {
  if (!h || !out) return SMR_E_INVALID_ARG;
  Ctx* c = &h->c;
  if (!check_scene(c)) return SMR_E_STATE;
  if (level < 0 || level >= c->nlev || (kind != 0 && kind != 1))
    return fail(c, SMR_E_INVALID_ARG, "level or kind out of range");
  if (c->spec_prec < 0) return fail(c, SMR_E_STATE, "no product has run yet");
  Level& L = c->lev[level];
  size_t elems = (size_t)L.nbox * L.K * 4 * c->spec_R;
  if (n_doubles < 2 * elems) return fail(c, SMR_E_INVALID_ARG, "output buffer too small");
  const void* src = kind == 0 ? L.d_out : L.d_in;
  cudaDeviceSynchronize();
  if (c->spec_prec == SMR_PREC_FP64) {
    SMR_CUDA(c, cudaMemcpy(out, src, elems * sizeof(double2), cudaMemcpyDeviceToHost));
  } else {
    std::vector<float2> t(elems);
    SMR_CUDA(c, cudaMemcpy(t.data(), src, elems * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < elems; ++i) { out[2 * i] = t[i].x; out[2 * i + 1] = t[i].y; }
  }
  return SMR_OK;
}

}  // extern "C"
