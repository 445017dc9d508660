// Internal interface between the host API (pw_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "pw_cx.cuh"
#include "../../include/pw.h"

namespace pw {

// One (E, k_par) point of a sweep batch.
struct PointDesc {
  double E;
  int kset;     // k-set slot holding its eigenvalues and overlaps
  int nL, nR;   // open channels of the left / right electrode
  int out;      // index into the caller's output arrays
  int skip;     // 1: threshold point, write NaN and do nothing else
  int N;        // device slices of the point's problem
  int dz_off;   // start of its dz[0..N+1] in the dz array
  long long en_off;   // its slice 0 in the eigenvalue array (units of n)
  long long o_off;    // its interface 0 in the overlap array (units of n*n)
  long long st_off;   // its interface 0 in the per-interface stores (Zst, Ust, LUst, PIVst, Fr, Gr)
  long long x_off;    // its slice 0 in the per-slice amplitudes (Xa, Xb)
};

// Descriptor of a point of a one-problem context: slices and interfaces of
// k-set `kset` at the uniform stride N+2 / N+1, stores of batch index `i`.
inline PointDesc make_point(double E, int kset, int nL, int nR, int out, int skip, int N, int i) {
  PointDesc d;
  d.E = E;
  d.kset = kset;
  d.nL = nL;
  d.nR = nR;
  d.out = out;
  d.skip = skip;
  d.N = N;
  d.dz_off = 0;
  d.en_off = (long long)kset * (N + 2);
  d.o_off = (long long)kset * (N + 1);
  d.st_off = (long long)i * (N + 1);
  d.x_off = (long long)i * (N + 2);
  return d;
}

// Geometry shared by the potential kernels.
struct WellSet {
  const double *xyz;     // 3 per well (slices) or 2 per well (leads)
  const double *v0;
  const double *sigma;
  int n;
};

struct TableArgs {
  zc *tab;               // (N+2) x tsz
  int nq, Dm, Dn;
  double b1x, b1y, b2x, b2y, area;
  const double *z_edges; // N+1
  WellSet slices;        // wells of the device region
  WellSet lead[2];       // electrode wells (x, y)
  double period[2];
  int explicit_slices;   // 1: slices 1..N were uploaded, skip them
  int explicit_lead[2];
};

struct SweepArgs {
  const PointDesc *pts;
  const double *En;      // kset slots: [kset][q][n], q = 0..N+1
  const zc *O;           // kset slots: [kset][p][n*n], p = 0..N
  const cc *O32;         // null, or FP32 copies of O (same layout and slots), read by the FP32 kernels
  const cc *O32t;        // null, or the same transposed (element (l, j) at j + l n), for the tensor-core B
  const double *dz;      // N+2: dz[0] = 0 (left lead), dz[1..N], dz[N+1] = 0
  void *R;               // per point n*n  (cx<T>)
  void *M;               // per point n*(2n+nc)  (cx<T>)
  int *piv;              // per point n
  int *status;           // per point
  double *T;             // caller outputs (by PointDesc.out)
  zc *t;
  int *nopen;
  double *err;
  int n, N, nc;          // N: the most slices of any point of the launch
  int p;                 // current interface (set by launch_sweep_batched)
  int panel_smem;        // LU panels staged in shared memory (set by launch_sweep_batched)
  void *Zst;             // FP32 sweep with refinement: per point (N+1) x n x n  (Z_p)
  void *Ust;             // per point (N+1) x n x nc  (u_p)
  void *LUst;            // per point (N+1) x n x n  (LU factors of W_p)
  int *PIVst;            // per point (N+1) x n      (row swaps of W_p)
  void *KV;              // per point 3 x n: 1/k^p, k^{p+1}, E+ of the current interface
  int mirror;            // 1: the z-mirrored transposed problem (slice q -> N+1-q,
                         //    overlap O_p -> O_{N-p}^T), used by the adjoint
  int wy_pairs;          // 1: points 2i and 2i+1 share overlaps and slice count (the
                         //    tensor-core [W|Y] then stages one B tile for both)
  int lapack_piv;        // set by the sweep: 1 in the tensor-core FP32 form, where each
                         //    panel's row swaps also reach the L columns left of it (so
                         //    the stored factors satisfy P W = L U with P from piv in
                         //    order) and the right-hand sides are eliminated after the LU
  int *rowexp;           // null, or per point 2n: the power-of-two row scales of R and of
                         //   R K_p^{-1} for the FP16-split [W|Y] (sweep variant bit 2)
  // separable nonlocal terms (FP64 sweep, pw_transmission_nonlocal): the particular
  // solutions' mode-space values at each slice's left (nl_fa) and right (nl_fb) edge,
  // [x_off + q][alpha][n] per point (zero in the electrodes); their unit-coefficient
  // responses are carried as right-hand-side columns nl_c0 .. nl_c0 + nl_m - 1
  const zc *nl_fa, *nl_fb;
  int nl_m, nl_c0;
  // null, or per point (launch index): the largest ratio max|u_ii| / min|u_ii|
  // of the LU factors of W_p over the interfaces swept so far (FP32 sweep)
  float *pivratio;
};

// 1 when every pair of points (2i, 2i+1) of a launch shares its overlaps and
// slice count (wy_pairs of SweepArgs).
inline int points_pair_up(const PointDesc *pd, int npts) {
  for (int i = 0; i + 1 < npts; i += 2)
    if (pd[i].o_off != pd[i + 1].o_off || pd[i].N != pd[i + 1].N) return 0;
  return 1;
}

// How the FP32 sweep of a variant stores the row swaps of its LU factors
// (piv_order of RefineArgs): the tensor-core form (bit 1) factors panels in
// pairs, or with LAPACK-ordered pivots when bit 3 is set too.
inline int stored_piv_order(int variant) { return (variant & 10) == 10 ? 1 : (variant & 2) ? 2 : 0; }

// Buffers of the FP64 refinement around the FP32 sweep (pw_refine.cu).
struct RefineArgs {
  const PointDesc *pts;
  const double *En;
  const zc *O;
  const cc *O32;         // null, or FP32 copies of O (the FP32 preconditioner passes read these)
  const cc *O32lo;       // null, or the FP32 remainders O - O32 (the double-float residual reads O32 + O32lo)
  const double *dz;
  const cc *Zst;         // per point (N+1) x n x n
  cc *Ust;               // per point (N+1) x n x nc
  const cc *LUst;        // per point (N+1) x n x n
  const int *PIVst;      // per point (N+1) x n
  cc *M;                 // per point n x (n + nc)
  int *piv;
  int *status;
  zc *Xa, *Xb;           // per point (N+2) x n x nc amplitudes (FP64)
  zc *Fr, *Gr;           // per point (N+1) x n x nc residuals (FP64)
  zc *carry;             // per point n x nc
  cc *tmp;               // per point 2n x nc
  double *corr;          // per point: relative size of the last correction of a_{N+1}
  double *corr_prev;     // per point: the same for the pass before
  double *T;
  zc *t;
  int *nopen;
  double *err;
  int n, N, nc;          // N: the most slices of any point
  long long x_slots;     // sum over points of N+2 (the Xa, Xb slots)
  long long st_slots;    // sum over points of N+1 (the Fr, Gr slots)
  int piv_order;         // how the stored LU factors hold their row swaps (the order
                         //    argument of cta_lu_replay): 0 each panel's swaps reach only
                         //    the columns right of it; 1 P W = L U (the tensor-core FP32
                         //    form with 128-row blocks); 2 panels in pairs (the
                         //    tensor-core FP32 form's default); see stored_piv_order
  uint16_t *Osl, *Ysl;   // null, or the residual's exact slices (BF16 bit patterns, K-contiguous):
                         //   RS_SLICES x 2n x 2n and RS_SLICES x (2 nc npts) x 2n, when every
                         //   point shares its overlaps (the residual products run on the tensor cores)
  int *Oexp, *Yexp;      //   their per-row / per-column power-of-two exponents (2n, 2 nc npts)
  double *Yacc;          //   the products O y of all points, column-major 2n x (2 nc npts)
  cc *Bw, *Yw;           // null, or n x (2 nc npts) each: when every point shares its overlaps
                         //   and slice count, the backward pass's O products of all points
                         //   run as one tensor-core GEMM (operands Bw, result Yw)
};

constexpr int RS_SLICES = 7;   // slices per operand of the tensor-core residual
constexpr int RS_BITS = 7;     // bits per slice
constexpr int RS_PAIRS = RS_SLICES * (RS_SLICES + 1) / 2;   // slice pairs with s + t < RS_SLICES
// bytes of the slice buffers for n basis functions and ncol = 2 nc npts columns
inline size_t rs_slice_bytes(int n, long long ncol) {
  return (size_t)RS_SLICES * 2 * n * (2 * (size_t)n + (size_t)ncol) * sizeof(uint16_t);
}

// 1 when every point of a launch has the same overlaps and slice count.
inline int points_share_overlaps(const PointDesc *pd, int npts) {
  for (int i = 1; i < npts; ++i)
    if (pd[i].o_off != pd[0].o_off || pd[i].N != pd[0].N) return 0;
  return npts > 0;
}

// Backward pass of a stored FP64 sweep (pw_grad.cu)
struct GradArgs {
  const PointDesc *pts;
  const double *En;
  const zc *O;
  const double *dz;
  const zc *Zst;         // per point (N+1) x n x n
  const zc *Ust;         // per point (N+1) x n x nc
  zc *Xa, *Xb;           // per point (N+2) x n x nc amplitudes
  zc *carry;             // per point n x nc
  zc *tmp;               // per point 2n x nc
  const int *status;
  int n, N, nc, mirror;
  const zc *nl_fa;       // null, or the particular solutions' left-edge values (as in SweepArgs):
  int nl_m, nl_c0;       //   columns nl_c0.. get b_p = Q a_q + P (e_q b_q + fa_q)
};

// Accumulation of the adjoint's eigenbasis matrices and their folding
struct GammaArgs {
  const PointDesc *pts;  // the original problem's descriptors
  const double *En;
  const double *dz;
  const zc *Xa, *Xb;     // original problem, left incidence
  const zc *Xa_m, *Xb_m; // mirrored transposed problem
  const int *status, *status_m;
  const double *weight;  // per point of the batch, or null
  zc *Gam;               // [slot][p-1][n x n], p = 1..N
  zc *gtab;              // [p-1][(2Dm+1)(2Dn+1)]
  int n, N, nc, npts;
};

// backward pass over interfaces p_hi down to p_lo (init: clear the amplitudes
// and the carry and set the incident a_0 first; the carry links calls that
// cover consecutive ranges from the right)
cudaError_t launch_grad_backward(const GradArgs &g, int npts, cudaStream_t s, int p_hi, int p_lo, bool init);
// Gamma_p and its fold onto the Fourier-table grid for the device slices
// p0 .. p0 + cnt - 1 (1-based) of k-set `slot`; Gam and T1 hold cnt matrices
cudaError_t launch_grad_gamma(const GammaArgs &h, int slot, int p0, int cnt, cudaStream_t s);
cudaError_t launch_grad_fold(const GammaArgs &h, int slot, int p0, int cnt, const zc *U, zc *T1, const int *mn, int Dm,
                             int Dn, cudaStream_t s);
cudaError_t launch_grad_wells(const GammaArgs &h, const WellSet &w, const double *z_edges, const double *b,
                              double area, int Dm, int Dn, double *dV0, const double *rate, double *dshift,
                              cudaStream_t s);
// separable nonlocal terms (pw_nonlocal.cu)
constexpr int kNlMaxProj = 8;    // projectors
constexpr int kNlMaxQuad = 32;   // Gauss-Legendre nodes per slice
constexpr int kNlMaxOpen = 64;   // open channels of the left electrode
struct NonlocalArgs {
  const PointDesc *pts;
  const double *En;      // kset slots [kset][q][n]
  const double *dz;      // N+2
  const double *zedge;   // N+1 slice edges z_0 .. z_N
  const zc *V;           // [kset][p = 1..N][alpha][n]: U_p^H amp_alpha (the projectors in mode space)
  const double *proj;    // per projector: tau_z, sigma, z_lo, z_hi
  const double *gl;      // Gauss-Legendre nodes and weights on [-1, 1]: x[q], w[q]
  int q;                 // nodes per slice
  zc *FA, *FB, *HA, *HB; // [x_off + q][alpha][n] (FA, FB: the particular solutions' edge values;
                         //   HA, HB: <W_beta| e^{ik(z - z_a)}>, <W_beta| e^{ik(z_b - z)}> per mode)
  zc *PP;                // [x_off + q][beta][alpha]: <W_beta | U f_alpha> of slice q
  const zc *Xa, *Xb;     // amplitudes of the stored sweep's backward pass (as in GradArgs)
  const zc *D;           // m x m coupling, row-major D[beta * m + alpha]
  double area;
  const int *status;
  double *T;             // caller output (by PointDesc.out)
  zc *C;                 // caller output or null: [out][alpha][channel], m x n_open^L per point
  int n, N, nc, m, c0, ks_N;
};
// V of one k-set slot: U_p^H amp_alpha for the device slices (grid N x m)
cudaError_t launch_nl_project(const zc *U, zc *V, const int *mn_unused, const double *G, double kx, double ky,
                              const double *tau_xy_sigma, double area, int n, int N, int m, cudaStream_t s);
cudaError_t launch_nl_slice_terms(const NonlocalArgs &a, int npts, cudaStream_t s);
cudaError_t launch_nl_solve(const NonlocalArgs &a, int npts, cudaStream_t s);
// the source columns of one interface step (FP64 sweep): Tacc_src += Y fa_q + fb_p
cudaError_t launch_nl_sources(const SweepArgs &a, int npts, int p, cudaStream_t s);

// periodic electrodes (pw_bands.cu)
struct BandArgs {
  int n, nprob;
  const zc *S;           // [prob][4][n*n]: S11, S12, S21, S22 of one electrode period
  const double *Eref;    // [prob][n]: eigenvalues of the electrode's reference slice
  const zc *Uref;        // [prob][n*n]: its modes
  int ref_shared;        // 1: one reference slice (Eref, Uref) for every problem
  const double *E;       // [prob]
  zc *work;              // [prob][band_work_elems(n)]
  int *ipiv;             // [prob][2n]
  int *keys;             // [prob][8n]
  zc *states;            // [prob][4][n*n]: aR, bR (right-going), aL, bL (left-going)
  int *prop;             // [prob][2n]: 1 for propagating columns (right-going 0..n-1, left-going n..2n-1)
  int *status;           // [prob]: 0 ok, 1 singular Cayley matrix, 2 no Schur form, 3 state counts, 4 band edge
};
__host__ __device__ size_t band_work_elems(int n);
cudaError_t launch_cbands(const BandArgs &a, cudaStream_t s);
struct PeriodicArgs {
  int n;
  const zc *Sdev;        // [pt][4][n*n]: S of [left reference slice, device, right reference slice]
  const zc *statesL, *statesR;   // [pt][4][n*n] as BandArgs.states
  const int *propL, *propR;      // [pt][2n]
  const int *bad;        // [pt]: nonzero when either electrode's states failed
  zc *work;              // [pt][periodic_work_elems(n)]
  int *ipiv;             // [pt][2n]
  double *T;             // caller output at index out[pt]
  const int *out;
};
size_t periodic_work_elems(int n);
cudaError_t launch_periodic_solve(const PeriodicArgs &a, int npts, cudaStream_t s);
cudaError_t launch_tilt_modes(const zc *U, zc *Ut, const double *G, double ax, double ay, int n, int count,
                              cudaStream_t s);
cudaError_t schur_selftest(zc *A, zc *Z, zc *v, int N, int sel, int *keys, int *out);

cudaError_t launch_grad_leads(const GammaArgs &h, const zc *U_all, const double *G, zc *scr,
                              const double rate[2][2], double *out, cudaStream_t s);

// potential tables and slice Hamiltonians
void launch_tables(const TableArgs &a, cudaStream_t s);
void launch_assemble_h(zc *H, const zc *tab, const int *mn, const double *G, double kx, double ky,
                       int n, int nq, int Dm, int Dn, cudaStream_t s);
// batched Hermitian eigensolver: H (in) -> U (out, same buffer); V scratch of
// the same size; status: Jacobi sweeps per matrix (negative: not converged)
// double_float: the mixed form's double-float solver; ws (ws_bytes >=
// heev_ws_bytes(n, 1), else null) lets its QL recurrence run in double-float
// as a separate launch over groups of as many matrices as the workspace holds
// tail: the launch is a partial last wave run on a side stream (timed as its
// own kernel kind); remap_last >= 0 (FP64 solver): the grid's last CTA takes
// matrix remap_last (relative to HU) instead of matrix nmat - 1
void launch_eig(zc *HU, zc *V, double *En, int *status, int n, int nmat, cudaStream_t s,
                bool double_float = false, void *ws = nullptr, size_t ws_bytes = 0, bool tail = false,
                int remap_last = -1);
size_t heev_ws_bytes(int n, int nmat);
// CTAs of the FP64 eigensolver resident on one SM at once (order n)
int heev_resident_per_sm(int n);
// FP32 copies of `count` n x n overlaps, plain, (when O32t is not null)
// transposed: O32t[j + l n] = O[l + j n], and (when O32lo is not null) the FP32
// remainders O - O32 (O32 + O32lo is O as a double-float)
void launch_overlaps_fp32(const zc *O, cc *O32, cc *O32t, cc *O32lo, int n, int count, cudaStream_t s);
// O_p = U_p^H U_{p+1}, p = 0..nq-2, for nslots consecutive k-set slots;
// double_float: accumulate in double-float (48-bit) on the FP32 pipe.  Pairs
// g = slot (nq-1) + p in [g0, g1) only (g1 < 0: all of them).
void launch_overlaps(const zc *U, zc *O, int n, int nq, int nslots, cudaStream_t s,
                     bool double_float = false, int g0 = 0, int g1 = -1);
// One interface step of the left-to-right sweep for every point of a batch,
// as a sequence of launches over (tiles x points).  variant bit 0: 512-thread
// CTAs with 128 x 64 GEMM tiles (else 256 threads, 64 x 64); bit 1 (FP32
// only): the [W|Y] product on the tcgen05 tensor cores (TF32 hi/lo split).
// sweep_variants: how many variants a precision has (0 .. count-1).
// wy0, wy1: optional events recorded around the [W|Y] GEMM launch.
// prepare_sweep_batched sets the kernels' shared-memory limits for n; call it
// before the first step of a size (and outside a stream capture).
cudaError_t prepare_sweep_batched(int n, int precision, int variant);
cudaError_t launch_sweep_batched(const SweepArgs &a, int npts, int p, int precision, cudaStream_t s,
                                 cudaEvent_t wy0 = nullptr, cudaEvent_t wy1 = nullptr, int variant = 0);
int sweep_batched_launches(int n, int precision, int variant);
int sweep_variants(int precision);
// the variants a batch times per N_G (the sweep's launch shapes; bit 4 only
// changes the refinement)
std::vector<int> sweep_variant_candidates(int precision);
// FP64 refinement of an FP32 sweep that stored Z_p, u_p and the LU factors:
// between min_iters and max_iters passes, stopping once every point's
// estimated remaining error of a_{N+1} (c_i^2 / c_{i-1} from the relative
// corrections c) is below tol; *passes = passes made
cudaError_t launch_refine(const RefineArgs &a, int npts, int min_iters, int max_iters, double tol,
                          cudaStream_t s, int *passes);
size_t refine_smem_bytes(int n);
// explicit interface S-matrices (FP64): npts CTAs, CTA b at point b and interface
// iface, or (by_iface) at point 0 and interface iface + b; output blocks at
// S + b * sstride (0: 4 n^2); mixed: the element (I11, I12, S21, S22) of Eq. recurrence2
cudaError_t launch_slice_smatrix(const PointDesc *pts, const double *En, const zc *O, const double *dz,
                                 zc *work, int *piv, int *status, zc *S, int n, int N, int iface,
                                 int npts, cudaStream_t s, int mixed = 0, size_t sstride = 0, int by_iface = 0);
// element strides (complex values) of the operands and result of a batched combination
struct Strides {
  size_t a, b, c;
};
// star products (FP64); CTA i combines Sa + i str.a and Sb + i str.b into Sab + i str.c
// (zero strides: 4 n^2 each)
cudaError_t launch_compose(const zc *Sa, const zc *Sb, zc *Sab, zc *work, int *piv, int *status,
                           int n, int npts, cudaStream_t s, Strides str = Strides{0, 0, 0});
// layer doubling with Eq. recurrence2 (FP64): one step per pair (work n x 4n per pair)
cudaError_t launch_compose_mixed(const zc *Ta, const zc *Tb, zc *Tab, zc *work, int *piv, int *status, int n,
                                 int npairs, cudaStream_t s, Strides str);
// Eq. scatter on mixed elements in place (work n x 3n per block)
cudaError_t launch_mixed_to_s(zc *T, size_t stride, zc *work, int *piv, int *status, int n, int nblocks,
                              cudaStream_t s);
// the 1-norm of each block's I11 (the switching measure of Eq. recurrence2)
cudaError_t launch_i11_norm(const zc *T, size_t stride, int n, int nblocks, double *out, cudaStream_t s);
// T of one point from its S11 and the electrodes' ascending eigenvalues
cudaError_t launch_t_from_s(const zc *S11, const double *EnL, const double *EnR, double E, int n, int nL, int nR,
                            double *T_out, cudaStream_t s);

// Read-only view of a one-problem context's geometry (pw_api.cu), for the
// batch executor (pw_batch.cu).
struct CtxView {
  int n, N, Dm, Dn, num_sms, precision, refine_iters;
  const zc *tab;         // device, (N+2) Fourier tables
  const int *mn;         // device, 2n
  const double *G;       // device, 2n
  const double *dz;      // host, N+2 (dz[0] = dz[N+1] = 0)
  cudaStream_t stream;
};
CtxView ctx_view(const pw_ctx *c);

// ---------------------------------------------------------------------------
// Per-kernel launch timing (pw_set_profiling).  While a profiled call runs on
// this host thread, g_ktimer points at the context's timer: every launch site
// below counts its launches by kind, and every `stride`-th launch of a kind is
// bracketed by CUDA events on the stream it is launched on.  With no timer set
// (the default, and inside every stream capture) the sites cost one test.
// ---------------------------------------------------------------------------
enum KernelKind : int {
  KK_VECTORS, KK_WY, KK_ROWEXP, KK_PANEL, KK_PANEL_APPLY, KK_TRAIL, KK_RHS_PERM, KK_FSDIAG, KK_FSUPD,
  KK_BSDIAG, KK_BSUPD, KK_FINISH,
  KK_REF_INIT, KK_REF_RESIDUAL, KK_RES_OSLICE, KK_RES_YSLICE, KK_RES_MM, KK_RES_FINISH, KK_REF_FWD_A,
  KK_REF_FWD_B, KK_REF_BWD_A, KK_REF_BWD_B, KK_REF_BWD_MM, KK_REF_BWD_C, KK_REF_FINISH,
  KK_TABLES, KK_ASSEMBLE, KK_HEEV, KK_QL, KK_ROT, KK_BACKT, KK_SORT, KK_OVERLAPS, KK_O32, KK_O32T,
  KK_HEEV_TAIL,
  KK_COUNT
};
const char *kernel_kind_name(int kind);
struct KernelTimer;
extern thread_local KernelTimer *g_ktimer;
// counts the launch; returns an event recorded on s when this launch is sampled
cudaEvent_t kt_begin(int kind, cudaStream_t s);
void kt_end(int kind, cudaEvent_t begin, cudaStream_t s);
// runs the launch statement(s) as one timed launch of `kind` on stream s
#define PW_TIMED(kind, s, ...)                                                                 \
  do {                                                                                         \
    const cudaEvent_t pw_kt_a_ = ::pw::g_ktimer ? ::pw::kt_begin((kind), (s)) : nullptr;        \
    __VA_ARGS__;                                                                               \
    if (::pw::g_ktimer) ::pw::kt_end((kind), pw_kt_a_, (s));                                    \
  } while (0)

constexpr double kThresholdRy = 1e-10;     // electrode channel at threshold
constexpr double kRefineTolRel = 1e-9;     // refinement stops below this estimated error of t

}  // namespace pw
