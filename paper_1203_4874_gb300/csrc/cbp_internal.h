// Internal (non-ABI) declarations shared by the libcbp translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include "cbp.h"

namespace cbp {

constexpr int kMaxN = 64;      // t1 + t2 (per-sample system width)
constexpr int kCnnSide = 256;  // learned proposal: network input side
constexpr int kCnnT = 15;      // learned proposal: kernel side
constexpr int kCnnParams = 19362;
constexpr int kMaxM = 32;      // samples per direction (scale system is 2M wide)
constexpr int kMaxRadixStages = 16;

// One frame batch as the kernels see it.
struct FrameDesc {
  const void* data;
  const uint64_t* tab;         // optional device table of per-frame base addresses
  int n, c, h, w;
  int f64;                     // 1: double elements, 0: float
  int64_t rs, cs, fs;          // row / channel / frame strides in elements
};

// Optional device tables of per-pair addresses (serving batches gather
// independent requests without copies): frames, kernels and latents.
struct PtrTables {
  const uint64_t* b1 = nullptr;
  const uint64_t* b2 = nullptr;
  const uint64_t* k1 = nullptr;
  const uint64_t* k2 = nullptr;
  const uint64_t* lat = nullptr;
};

// One Stockham stage of radix R: Ns = product of the earlier radices, Nr = N / R,
// magic multipliers mNs, mNr for exact division by Ns and Nr (0 encodes 1),
// and the offset of the stage's twiddles w_{Ns R}^{k r} (k < Ns, 1 <= r < R)
// in the plan's twiddle table.
struct FftStage {
  int R, Ns, Nr;
  uint32_t mNs, mNr;
  int tw;
};

// Mixed-radix FFT plan: N = prod of the stages' radices (9, 8, 7, 5, 4, 3, 2).
struct FftPlan {
  int n;
  int nst;
  int ntw;                     // twiddle-table entries (N - 1, at least 1)
  FftStage st[kMaxRadixStages];
};

// Everything one batched call needs: shapes, precisions, workspace layout.
struct Plan {
  int n, C;
  int H1, W1, H2, W2;          // blurred frame sizes
  int H, W;                    // latent size
  int t1, t2, M, ns, nn;       // ns = M/2 + 1 solved samples per direction; nn = t1 + t2
  int Ph, Pw, Pw2;             // FFT grid; Pw2 = Pw/2 + 1 stored spectrum columns
  int Pw2p;                    // row pitch of the spectra: Pw2 rounded up to a multiple of 4
  int mixed;                   // estimation path: 0 FP64, 1 mixed
  int fft_f64;                 // deconvolution arithmetic in double
  int frames_f64;              // float64 frames (fold bins are doubles, else (hi, lo) float pairs)
  int pz_all;                  // mixed path: double copies of every sample (stage outputs)
  int single_kernel;           // deconvolve B1 by K1 only
  int pw_half;                 // Pw even: real row FFTs via half-length complex FFTs
  int learned;                 // learned path: proposal + consistency gate first
  int col_strips;              // column strips of the column pass
  int col_fused;               // column pass computes the kernel spectra itself (no K^ buffer)
  int scale_mode;              // 0: two-order least squares, 1: k1-only, 2: support constraint
  double accept_rho;
  double eps;
  FftPlan fp_h, fp_w, fp_w2;   // plans of Ph, Pw, Pw/2
  // workspace layout (byte offsets into one device allocation)
  size_t off_pz2[2], off_pz1[2];   // cd [n][C][ns][len] sample polynomials (double)
  size_t off_pz2f[2], off_pz1f[2]; // cdf float-float copies for the mixed path's Gram
  size_t off_fbr[2], off_fbc[2];   // 8-byte [n][C][M][H_Bk] row / [n][C][M][W_Bk] column fold bins
  size_t off_x;                    // cd [n][2][ns][nn]
  size_t off_gall;                 // cd [n][2][ns][nn][nn] per-sample normal matrices
  size_t off_sdiag;                // double [n][2][ns][4]
  size_t off_resid;                // cd [n][2][ns][C][Lmax] (FP64 path residual scratch)
  int Lmax;
  size_t off_kd;                   // double [n][t1*t1 + t2*t2]
  size_t off_bad;                  // int [n] non-finite input flags
  size_t off_err;                  // int: set by a kernel whose copy did not complete in time
  size_t off_diag;                 // cbp_diag [n]
  size_t off_tw_h, off_tw_w;       // cpx<T_fft> twiddles exp(-2 pi i k / P), k < P
  size_t off_stw_h, off_stw_r;     // cpx<T_fft> stage twiddles of the column and row plans
  size_t off_tw2r, off_tw2c;       // float twiddles w_N^(a b) of the in-register passes, laid out
                                   // so a warp's lanes read consecutive entries (0: not used)
  size_t off_krow;                 // fused column pass: the kernels' row transforms R_k,p(v), float
                                   // complex [n][2][max(t1, t2)][Pw2p] (0: not used)
  size_t off_khat;                 // cpx<T_fft> [n][2][Ph][Pw2p] (learned gate, unfused column pass)
  size_t off_spec[2];              // cpx<T_fft> [n][C][H_Bk][Pw2p]
  size_t off_ihat;                 // cpx<T_fft> [n][C][H][Pw2p]
  size_t off_io_b[2], off_io_k[2], off_io_lat; // device staging for host I/O
  size_t off_cnn;                  // learned path: network workspace
  size_t off_acc;                  // int [n] proposal accepted
  size_t off_rho;                  // double [n] consistency residual of the proposal
  size_t off_rpart;                // double [n][C][col_strips][2] residual partial sums
  size_t total;
};

// Kernel-size scan of a batch (cbp_estimate_size): candidates t1' in
// [t_min, t_min + ncand), t2' = t1' - d; workspace layout.
struct SizePlan {
  int n, C, d, t_min, ncand;
  double tol;
  size_t off_rows[2], off_cols[2];   // cd [n][C][H_k] row sums, [n][C][W_k] column sums
  size_t off_ratio;                  // double [n][2][ncand] per order
  size_t off_rmax;                   // double [n][ncand] the larger of the two (-1: excluded)
  size_t off_t;                      // int [n][3]: t1, t2, found
  size_t total;
};

// ---- planning (cbp_plan.cpp) ----
int next_7_smooth(int n);
bool make_fft_plan(int n, FftPlan* p);
cbp_status make_plan(const cbp_frames* b1, const cbp_frames* b2, const cbp_params* prm,
                     Plan* plan);
cbp_status make_size_plan(const cbp_frames* b1, const cbp_frames* b2, const cbp_size_params* sp,
                          SizePlan* plan);
FrameDesc frame_desc(const cbp_frames* f, const void* data_override);

// ---- launchers (one per .cu file) ----
// A1: sample polynomials (cbp_eval.cu): the fold-only row pass, then the
// bins' M-point DFTs.  In a deblurring call the folds ride on the row FFT pass
// (launch_row_pass with fold and fft) and only launch_fold_dft follows.
void launch_eval(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                 cudaStream_t st);
void launch_fold_dft(const Plan& p, char* ws, cudaStream_t st);
// A2 + A3: per-sample Gram and null vector (cbp_solve.cu)
void launch_sample_solve(const Plan& p, char* ws, cudaStream_t st);
// A4 + A5: lift, scale fix, kernels (cbp_solve.cu)
void launch_scale_solve(const Plan& p, char* ws, void* k1_out, void* k2_out, int out_f64,
                        cudaStream_t st, const uint64_t* k1_tab = nullptr,
                        const uint64_t* k2_tab = nullptr);
// load caller kernels into the internal double buffer (CBP_FLAG_KERNELS_IN)
void launch_kernels_in(const Plan& p, char* ws, const void* k1, const void* k2, int in_f64,
                       cudaStream_t st, const uint64_t* k1_tab = nullptr,
                       const uint64_t* k2_tab = nullptr);
// A6: deconvolution (cbp_fft.cu)
void init_twiddles(const Plan& p, char* ws, cudaStream_t st);
void launch_kernel_spectra(const Plan& p, char* ws, cudaStream_t st);
// One read of every frame row: A1 folds (fold) and/or A6 forward row FFTs (fft).
void launch_row_pass(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                     cudaStream_t st, bool fold, bool fft);
// shared memory of the row pass at one row per group (the planner's limit check)
size_t row_pass_min_smem(const Plan& p);
void launch_col_deconv(const Plan& p, char* ws, cudaStream_t st);
// the fused column pass (cbp_colpass.cu): kernel spectra computed in the pass
bool col_pass_fused(const Plan& p);
void launch_col_deconv_fused(const Plan& p, char* ws, cudaStream_t st);
int fused_strips(const Plan& p);   // column strips of the fused column pass
// learned path, fused column pass: the proposal's deconvolution with the
// residual sums, then the per-pair decision
void launch_col_gate_fused(const Plan& p, char* ws, cudaStream_t st);
// per-pair consistency residual from `strips` partial sums per channel, and the decision
void launch_gate(const Plan& p, char* ws, cudaStream_t st, int strips);
void launch_row_ifft(const Plan& p, char* ws, void* latent, int out_f64, cudaStream_t st,
                     const uint64_t* lat_tab = nullptr);
// learned path: consistency residual of the kernels in kd (column pass in
// residual mode, then the per-pair gate: rho, accepted)
void launch_residual_gate(const Plan& p, char* ws, cudaStream_t st);
// checked builds: bytes the bulk-copy barriers over-expect (false in a normal build)
bool set_tx_extra(uint32_t bytes);
// learned proposal (cbp_cnn.cu)
size_t cnn_workspace(int n, bool train);
void cnn_forward(const FrameDesc& b1, const FrameDesc& b2, int n, const float* prm, char* ws,
                 cudaStream_t st, const cbp_cnn_trace* tr = nullptr, int* err = nullptr);
const float* cnn_kernels(char* ws, int n);
void cnn_to_kd(char* ws, int n, double* kd, cudaStream_t st);
void cnn_train_step(const FrameDesc& b1, const FrameDesc& b2, int n, const float* kt, float* prm,
                    float* m, float* v, const cbp_adamw& hp, float* loss, char* ws, cudaStream_t st,
                    const cbp_cnn_trace* tr = nullptr);
// Eq. 1 forward model (cbp_forward.cu)
void launch_forward_blur(const void* latent, int n, int c, int h, int w, int f64,
                         const double* kernel, int t, double sigma, uint64_t seed, void* out,
                         cudaStream_t st);
void launch_synth_latent(const double* blobs, int nblobs, int n, int c, int h, int w, int f64,
                         double floor_amp, uint64_t seed, void* out, cudaStream_t st);
// Section 3 multi-level security: LSB truncation of a frame buffer (cbp_forward.cu)
void launch_truncate_lsb(const void* in, int f64, int64_t count, int bits, int drop, void* out,
                         cudaStream_t st);
// camera side (Section 3): per-frame kernel draws (cbp_forward.cu) and one
// round of the coprimality test with the redraw decision (cbp_solve.cu)
void launch_draw_kernels(int n, int t, int kind, int frame0, uint64_t seed, const int* active,
                         const int* attempt, double* kd, cudaStream_t st);
void launch_coprime_round(const double* ka, const double* kb, int n, int ta, int tb, int M,
                          double tol, int max_attempts, int* active, int* attempt, int* pass,
                          int* any, cudaStream_t st);
// the solver's reciprocal routines, elementwise (verification)
void launch_check_recip(const double* x, int64_t n, double* r, double* q, cudaStream_t st);
size_t sample_solve_smem(int nn);
// kernel-size scan (cbp_solve.cu): plane sums, per-candidate ratios, the pick
void launch_size_scan(const SizePlan& sp, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                      cudaStream_t st);
size_t size_scan_smem();
size_t scale_solve_smem(int M, int nn);

}  // namespace cbp
