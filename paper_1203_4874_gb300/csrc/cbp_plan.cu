// Host-side planning: argument validation, FFT factorisation and the layout of
// the per-call device workspace.
#include <algorithm>
#include <cmath>
#include "cbp_common.cuh"
#include "cbp_internal.h"

namespace cbp {

int next_7_smooth(int n) {
  for (int k = std::max(n, 1);; ++k) {
    int r = k;
    for (int p : {2, 3, 5, 7})
      while (r % p == 0) r /= p;
    if (r == 1) return k;
  }
}

static uint32_t magic_div(int d) {
  return d <= 1 ? 0u : (uint32_t)(((uint64_t(1) << 32) + (uint64_t)d - 1) / (uint64_t)d);
}

bool make_fft_plan(int n, FftPlan* p) {
  if (n < 1) return false;
  p->n = n;
  p->nst = 0;
  // radices, largest first; then an odd radix moved to the front: the first
  // stage writes its outputs R elements apart, and an odd stride keeps those
  // shared-memory stores free of bank conflicts
  int radix[kMaxRadixStages];
  int nr = 0;
  for (int r = n; r > 1;) {
    int R = 0;
    for (int cand : {9, 8, 7, 5, 4, 3, 2})
      if (r % cand == 0) {
        R = cand;
        break;
      }
    if (!R || nr >= kMaxRadixStages) return false;
    radix[nr++] = R;
    r /= R;
  }
  for (int i = 0; i < nr; ++i)
    if (radix[i] & 1) {
      const int R = radix[i];
      for (int j = i; j > 0; --j) radix[j] = radix[j - 1];
      radix[0] = R;
      break;
    }
  int Ns = 1, off = 0;
  for (int i = 0; i < nr; ++i) {
    const int R = radix[i];
    FftStage& st = p->st[p->nst++];
    st.R = R;
    st.Ns = Ns;
    st.Nr = n / R;
    st.mNs = magic_div(Ns);
    st.mNr = magic_div(st.Nr);
    st.tw = off;
    off += Ns * (R - 1);
    Ns *= R;
  }
  p->ntw = off > 0 ? off : 1;
  return true;
}

static bool valid_frames(const cbp_frames* f) {
  if (!f || !f->data || f->n < 1 || f->c < 1 || f->h < 1 || f->w < 1) return false;
  if (f->dtype != CBP_F32 && f->dtype != CBP_F64) return false;
  const int64_t rs = f->row_stride ? f->row_stride : f->w;
  const int64_t cs = f->chan_stride ? f->chan_stride : (int64_t)f->h * rs;
  const int64_t fs = f->frame_stride ? f->frame_stride : (int64_t)f->c * cs;
  if (rs < f->w || cs < (int64_t)(f->h - 1) * rs + f->w) return false;
  if (f->n > 1 && fs < (int64_t)(f->c - 1) * cs + (int64_t)(f->h - 1) * rs + f->w) return false;
  return true;
}

FrameDesc frame_desc(const cbp_frames* f, const void* data_override) {
  FrameDesc d;
  d.data = data_override ? data_override : f->data;
  d.tab = nullptr;
  d.n = f->n;
  d.c = f->c;
  d.h = f->h;
  d.w = f->w;
  d.f64 = f->dtype == CBP_F64;
  d.rs = f->row_stride ? f->row_stride : f->w;
  d.cs = f->chan_stride ? f->chan_stride : (int64_t)f->h * d.rs;
  d.fs = f->frame_stride ? f->frame_stride : (int64_t)f->c * d.cs;
  return d;
}

static bool is_7_smooth(int n) { return n >= 1 && next_7_smooth(n) == n; }

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

cbp_status make_plan(const cbp_frames* b1, const cbp_frames* b2, const cbp_params* prm,
                     Plan* P) {
  if (!prm || !valid_frames(b1) || !valid_frames(b2)) return CBP_ERR_INVALID_ARG;
  if (b1->n != b2->n || b1->c != b2->c || b1->dtype != b2->dtype) return CBP_ERR_INVALID_ARG;
  if (prm->path != CBP_PATH_FP64 && prm->path != CBP_PATH_MIXED && prm->path != CBP_PATH_LEARNED)
    return CBP_ERR_INVALID_ARG;
  if (!(prm->eps >= 0.0) || !std::isfinite(prm->eps)) return CBP_ERR_INVALID_ARG;
  const int t1 = prm->t1, t2 = prm->t2;
  if (t1 < 1 || t2 < 1) return CBP_ERR_INVALID_ARG;
  if (t1 + t2 > kMaxN) return CBP_ERR_UNSUPPORTED;
  Plan p = {};
  p.n = b1->n;
  p.C = b1->c;
  p.H1 = b1->h;
  p.W1 = b1->w;
  p.H2 = b2->h;
  p.W2 = b2->w;
  p.t1 = t1;
  p.t2 = t2;
  p.H = p.H1 - t1 + 1;
  p.W = p.W1 - t1 + 1;
  if (p.H < 1 || p.W < 1) return CBP_ERR_SIZE_MISMATCH;
  if (p.H2 != p.H + t2 - 1 || p.W2 != p.W + t2 - 1) return CBP_ERR_SIZE_MISMATCH;
  p.M = prm->m ? prm->m : std::max(t1, t2);
  if (p.M < std::max(t1, t2)) return CBP_ERR_INVALID_ARG;
  if (p.M > kMaxM) return CBP_ERR_UNSUPPORTED;
  p.ns = p.M / 2 + 1;
  p.nn = t1 + t2;
  const int hmax = std::max(p.H1, p.H2), wmax = std::max(p.W1, p.W2);
  p.Ph = prm->pad_h ? prm->pad_h : next_7_smooth(hmax);
  p.Pw = prm->pad_w ? prm->pad_w : next_7_smooth(wmax);
  if (p.Ph < hmax || p.Pw < wmax || !is_7_smooth(p.Ph) || !is_7_smooth(p.Pw))
    return CBP_ERR_INVALID_ARG;
  p.Pw2 = p.Pw / 2 + 1;
  p.Pw2p = (p.Pw2 + 3) & ~3;   // 32-byte rows for float spectra: a 4-column strip row is one sector
  p.pw_half = (p.Pw % 2 == 0) ? 1 : 0;
  p.mixed = prm->path != CBP_PATH_FP64;
  const int frame_f64 = b1->dtype == CBP_F64;
  p.fft_f64 = (frame_f64 && !p.mixed) ? 1 : 0;
  p.frames_f64 = frame_f64;
  p.single_kernel = (prm->flags & CBP_FLAG_SINGLE_KERNEL) ? 1 : 0;
  const bool k1_only = (prm->flags & CBP_FLAG_K1_ONLY) != 0;
  const bool support = (prm->flags & CBP_FLAG_SCALE_SUPPORT) != 0;
  if (k1_only && support) return CBP_ERR_INVALID_ARG;
  if (support && p.M <= std::max(t1, t2)) return CBP_ERR_INVALID_ARG;   // needs M > t
  p.scale_mode = k1_only ? 1 : support ? 2 : 0;
  if (k1_only) p.single_kernel = 1;            // the paper's division of B1 by K1
  p.learned = prm->path == CBP_PATH_LEARNED ? 1 : 0;
  if (p.learned && (t1 != kCnnT || t2 != kCnnT)) return CBP_ERR_UNSUPPORTED;  // network output size
  if (p.learned && !(prm->accept_rho >= 0.0)) return CBP_ERR_INVALID_ARG;
  p.accept_rho = prm->accept_rho;
  p.eps = prm->eps;
  if (!make_fft_plan(p.Ph, &p.fp_h) || !make_fft_plan(p.Pw, &p.fp_w)) return CBP_ERR_INVALID_ARG;
  if (p.pw_half && !make_fft_plan(p.Pw / 2, &p.fp_w2)) return CBP_ERR_INVALID_ARG;
  // shared-memory limits of the kernels
  const size_t smem_max = 227 * 1024;
  const size_t ce = p.fft_f64 ? 16 : 8;
  const size_t cw = p.fft_f64 ? 2 : 4;
  const size_t nrow = p.pw_half ? p.Pw / 2 : p.Pw;
  // row pass at one row per group; exact magic division needs rows * N < 2^16
  if (row_pass_min_smem(p) > smem_max || nrow > 16384) return CBP_ERR_UNSUPPORTED;
  if (3 * cw * ce * p.Ph > smem_max || cw * p.Ph > 65536) return CBP_ERR_UNSUPPORTED;
  if (sample_solve_smem(p.nn) > smem_max || scale_solve_smem(p.M, p.nn) > smem_max)
    return CBP_ERR_UNSUPPORTED;

  // workspace layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t n = p.n, C = p.C, ns = p.ns;
  p.off_pz2[0] = take(n * C * ns * p.H1 * 16);
  p.off_pz2[1] = take(n * C * ns * p.H2 * 16);
  p.off_pz1[0] = take(n * C * ns * p.W1 * 16);
  p.off_pz1[1] = take(n * C * ns * p.W2 * 16);
  if (p.mixed) {
    p.off_pz2f[0] = take(n * C * ns * p.H1 * 16);
    p.off_pz2f[1] = take(n * C * ns * p.H2 * 16);
    p.off_pz1f[0] = take(n * C * ns * p.W1 * 16);
    p.off_pz1f[1] = take(n * C * ns * p.W2 * 16);
  }
  for (int k = 0; k < 2; ++k) {
    p.off_fbr[k] = take(n * C * (size_t)p.M * (k ? p.H2 : p.H1) * 8);
    p.off_fbc[k] = take(n * C * (size_t)p.M * (k ? p.W2 : p.W1) * 8);
  }
  p.off_x = take(n * 2 * ns * p.nn * 16);
  p.off_gall = take(n * 2 * ns * (size_t)p.nn * p.nn * 16);
  p.off_sdiag = take(n * 2 * ns * 4 * 8);
  p.Lmax = std::max(p.H1, p.W1) + t2 - 1;
  const size_t resid = n * 2 * ns * C * (size_t)p.Lmax * 16;
  const size_t abytes = n * 4 * (size_t)p.M * p.M * 16;
  p.off_resid = take(std::max(resid, abytes));
  p.off_kd = take(n * (size_t)(t1 * t1 + t2 * t2) * 8);
  p.off_bad = take(n * 4);
  p.off_err = take(4);
  p.off_diag = take(n * sizeof(cbp_diag));
  p.off_tw_h = take(p.Ph * ce);
  p.off_tw_w = take(p.Pw * ce);
  p.off_stw_h = take((size_t)p.fp_h.ntw * ce);
  p.off_stw_r = take((size_t)(p.pw_half ? p.fp_w2.ntw : p.fp_w.ntw) * ce);
  p.col_fused = col_pass_fused(p) ? 1 : 0;
  // [k2][n1] and [n1][k2] of w_972^(n1 k2) (row passes); [m][n1] and [p][k2] of w_1120 (column pass)
  p.off_tw2r = (!p.fft_f64 && p.pw_half && p.fp_w2.n == 972) ? take(2 * 972 * 8) : 0;
  p.off_tw2c = p.col_fused ? take(2 * 1120 * 8) : 0;
  p.off_krow = p.col_fused ? take(n * 2 * (size_t)std::max(t1, t2) * p.Pw2p * 8) : 0;
  if (!p.col_fused) p.off_khat = take(n * 2 * (size_t)p.Ph * p.Pw2p * ce);
  p.off_spec[0] = take(n * C * (size_t)p.H1 * p.Pw2p * ce);
  p.off_spec[1] = take(n * C * (size_t)p.H2 * p.Pw2p * ce);
  p.off_ihat = take(n * C * (size_t)p.H * p.Pw2p * ce);
  p.col_strips = (p.Pw2 + (int)cw - 1) / (int)cw;
  if (p.learned) {
    p.off_cnn = take(cnn_workspace(p.n, false));
    p.off_acc = take(n * 4);
    p.off_rho = take(n * 8);
    const int strips = p.col_fused ? fused_strips(p) : p.col_strips;
    p.off_rpart = take(n * C * (size_t)strips * 2 * 8);
  }
  if (prm->flags & CBP_FLAG_HOST_IO) {
    const size_t es = frame_f64 ? 8 : 4;
    p.off_io_b[0] = take(n * C * (size_t)p.H1 * p.W1 * es);
    p.off_io_b[1] = take(n * C * (size_t)p.H2 * p.W2 * es);
    p.off_io_k[0] = take(n * (size_t)t1 * t1 * 8);
    p.off_io_k[1] = take(n * (size_t)t2 * t2 * 8);
    p.off_io_lat = take(n * C * (size_t)p.H * p.W * es);
  }
  p.total = off;
  *P = p;
  return CBP_OK;
}

cbp_status make_size_plan(const cbp_frames* b1, const cbp_frames* b2, const cbp_size_params* sp,
                          SizePlan* P) {
  if (!valid_frames(b1) || !valid_frames(b2)) return CBP_ERR_INVALID_ARG;
  if (b1->n != b2->n || b1->c != b2->c || b1->dtype != b2->dtype) return CBP_ERR_INVALID_ARG;
  // full convolution: both blurred sizes differ by t1 - t2
  const int d = b1->h - b2->h;
  if (b1->w - b2->w != d) return CBP_ERR_SIZE_MISMATCH;
  SizePlan p = {};
  p.n = b1->n;
  p.C = b1->c;
  p.d = d;
  const int lo_valid = std::max(1, d + 1);                 // t2' = t1' - d >= 1
  int hi_valid = std::min(b1->h, b1->w);                   // a latent of at least one pixel
  hi_valid = std::min(hi_valid, (kMaxN + d) / 2);          // t1' + t2' <= kMaxN
  p.t_min = std::max(sp && sp->t_min > 0 ? sp->t_min : 1, lo_valid);
  const int t_max = std::min(sp && sp->t_max > 0 ? sp->t_max : 32, hi_valid);
  if (t_max < p.t_min) return CBP_ERR_INVALID_ARG;
  p.ncand = t_max - p.t_min + 1;
  p.tol = sp && sp->tol > 0.0 ? sp->tol : 1e-6;
  if (!std::isfinite(p.tol)) return CBP_ERR_INVALID_ARG;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t n = p.n, C = p.C;
  p.off_rows[0] = take(n * C * (size_t)b1->h * 16);
  p.off_rows[1] = take(n * C * (size_t)b2->h * 16);
  p.off_cols[0] = take(n * C * (size_t)b1->w * 16);
  p.off_cols[1] = take(n * C * (size_t)b2->w * 16);
  p.off_ratio = take(n * 2 * (size_t)p.ncand * 8);
  p.off_rmax = take(n * (size_t)p.ncand * 8);
  p.off_t = take(n * 3 * sizeof(int));
  p.total = off;
  *P = p;
  return CBP_OK;
}

}  // namespace cbp
