/*
 * pw.h -- C ABI of the GB300 plane-wave multiple-scattering transport library.
 *
 * The library computes, for a slice model of a junction between two
 * electrodes (z-invariant, or z-periodic through pw_set_periodic_electrode),
 * the transmission T(E, k_par) = Tr(t^H t) of Li, Chu,
 * Zhang & Cheng, "Electron transport in graphene/graphene side-contact junction
 * by plane-wave multiple scattering method" (PRB 2015):
 *   - Sec. II A / Eq. loc: 2D plane-wave basis {G_perp}, slice Hamiltonians
 *     H_p(G,G') = |k+G|^2 delta + V^p(G-G') and their eigenmodes;
 *   - App. A Eqs. transfer and scatter: the interface scattering matrix S(p,p+1);
 *   - Eq. recurrence: the star product (layer doubling) of scattering matrices;
 *   - App. C with z-invariant electrodes (slices 0 and N+1): t = S11(0,N+1)
 *     on open channels, flux-normalised, and T = Tr(t^H t).
 * Units: Rydberg atomic units (hbar^2/2m = 1, bohr, Ry).
 *
 * Conventions for every entry point
 *   - All calls return a pw_status.  The first failure inside a context is
 *     latched: later calls on that context return it until pw_destroy.
 *   - Arguments named *_dev are device pointers (CUDA global memory of the
 *     context's device), written asynchronously on the context's stream; all
 *     other pointers are host pointers read before the call returns.
 *   - The caller owns every input and output buffer; the context owns its
 *     workspaces and frees them in pw_destroy.  No C++ exception crosses the ABI.
 *   - Complex numbers are interleaved (re, im) doubles, i.e. C99 double _Complex.
 *   - Matrices are column-major n x n blocks (element (i,j) at i + j*n).
 *   - Channel order: the eigenmodes of every slice and electrode are sorted by
 *     ascending eigenvalue E_n; the open channels of an electrode at energy E
 *     are therefore its first n_open modes.
 */
#ifndef PW_H
#define PW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pw_ctx pw_ctx;
typedef struct pw_batch pw_batch;

typedef enum {
  PW_OK = 0,
  PW_EINVAL = 1,      /* bad argument or descriptor */
  PW_ENOMEM = 2,      /* device allocation failed */
  PW_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  PW_ESINGULAR = 4,   /* zero pivot in an LU factorisation */
  PW_ETHRESH = 5,     /* |E - E_n| < 1e-10 Ry for an electrode channel (k_n = 0) */
  PW_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  PW_ENOTCONV = 7     /* the slice eigensolver did not converge */
} pw_status;

typedef struct { double re, im; } pw_c128;

/* Arithmetic of the path.  PW_FP64: every step in FP64.  PW_MIXED_FP32: the
 * slice eigenmodes and the overlaps in FP64 (or, with launch variant bit 5, in
 * double-float: a value is the sum of two FP32 numbers, 48 significant bits,
 * on the FP32 pipe), the star-product sweep
 * in FP32 (its GEMMs on the tensor cores as TF32 hi/lo products), then passes
 * of iterative refinement of the whole interface-matching system whose
 * residuals are formed in double-float (with launch variant bit 4, as exact
 * BF16 slice products on the tensor cores when all points of a launch share
 * one k_par and N_G is a multiple of 4 up to 512) until the estimated
 * remaining error of t falls below 1e-9 relative; T and t are accumulated in
 * FP64. */
enum { PW_FP64 = 0, PW_MIXED_FP32 = 1 };

/*
 * Problem description (Sec. II A).  The transverse cell is spanned by a1, a2
 * (bohr); the basis is every G = m b1 + n b2 with |G|^2 <= ecut (whole shells)
 * or, if ng_exact > 0, the first ng_exact G ordered by (|G|^2, m, n), with
 * |G|^2 grouped into shells at 1e-8 Ry.  The device region is cut into
 * n_slices slices by the increasing z_edges[0..n_slices] (bohr).
 *
 * Potential of slice p (Eq. loc, the slice average of V_loc): either
 *   - n_wells Gaussian wells V(r) = -v0 exp(-|r - R|^2 / (2 sigma^2)), centres
 *     well_xyz[3*i + {0,1,2}] = (x, y, z) with z along transport, averaged over
 *     the slice thickness in closed form, or
 *   - explicit Fourier tables slice_vg (non-NULL overrides the wells): for each
 *     slice, (2*Dm+1) x (2*Dn+1) values V^p(dm b1 + dn b2) stored row-major
 *     [p][dm + Dm][dn + Dn], with (Dm, Dn) = vg_half.  Tables must satisfy
 *     V(-dG) = conj(V(dG)) (a real potential) and cover every G - G'.
 * Electrodes (slices 0 and N+1, App. C with z-invariant leads): either the
 * z-average over lead_period of lead_n_wells wells at transverse positions
 * lead_well_xy (0 wells = the V = 0 electrode), or an explicit table lead_vg
 * (same layout, one table).
 */
typedef struct {
  double a1[2], a2[2];
  double ecut;
  int ng_exact;
  int n_slices;
  const double *z_edges;
  int n_wells;
  const double *well_xyz;
  const double *well_v0;
  const double *well_sigma;
  int lead_n_wells[2];
  const double *lead_well_xy[2];
  const double *lead_well_v0[2];
  const double *lead_well_sigma[2];
  double lead_period[2];
  int vg_half[2];
  const pw_c128 *slice_vg;
  const pw_c128 *lead_vg[2];
  int precision;               /* PW_FP64 or PW_MIXED_FP32 */
  int refine_iters;            /* PW_MIXED_FP32 only: the most FP64 refinement
                                  passes (at least min(2, this) are made; more
                                  stop once every point's estimated remaining
                                  relative error of t, c_i^2 / c_{i-1} from the
                                  sizes c of successive corrections, is below
                                  1e-9); 0 = default (4), -1 = none */
  /* Motion of the geometry with one scalar parameter theta (for the side-
   * contact junction: the sheet gap, each sheet moving by half of it), used
   * only by pw_grad's dgap_host.  Transverse displacement per unit theta
   * (bohr per bohr, x then y):
   *   well_shift_rate   host, 2 per device well, or NULL (wells fixed)
   *   lead_shift_rate   left then right electrode; the electrode potential is
   *                     translated rigidly (its table becomes
   *                     e^{-i dG.delta} V(dG)) */
  const double *well_shift_rate;
  double lead_shift_rate[2][2];
} pw_setup_desc;

/* Builds the basis (Sec. II A) and uploads the slice geometry; the Fourier
 * tables V^p(dG) are evaluated on the device.  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream) on the current device.  On success *out owns
 * all device state of the problem. */
pw_status pw_setup(const pw_setup_desc *desc, void *cuda_stream, pw_ctx **out);

/* Frees every workspace of the context (synchronises its stream). */
void pw_destroy(pw_ctx *ctx);

/* Static text of a status code. */
const char *pw_status_str(pw_status s);

/* Latched status of the context (PW_OK if no call has failed). */
pw_status pw_get_error(const pw_ctx *ctx);
/* The first failing CUDA runtime call behind a latched PW_ECUDA / PW_ENOMEM:
 * "<cudaError name> at <source>:<line>" (empty when none), NUL-terminated into
 * buf[len].  Setting PW_SYNC_CHECK=1 in the environment makes every stage
 * synchronise its stream, so an asynchronous kernel failure is reported by
 * the stage that launched it. */
pw_status pw_get_error_detail(const pw_ctx *ctx, char *buf, int len);

/* Basis size N_G and slice count N of the context (0 for NULL). */
int pw_ng(const pw_ctx *ctx);
int pw_n_slices(const pw_ctx *ctx);

/* Copies the basis as integer pairs (m, n) into mn_host[2*N_G] (host). */
pw_status pw_get_gvectors(const pw_ctx *ctx, int *mn_host);

/* Fourier tables of slices 0..N+1 (left electrode, slices 1..N, right
 * electrode) as (N+2) x (2*Dm+1) x (2*Dn+1) complex values, row-major, into
 * vg_dev; (Dm, Dn) = twice the largest |m|, |n| of the basis, returned in
 * half_host[2].  Sec. II A (slice-averaged V_loc). */
pw_status pw_potential_tables(pw_ctx *ctx, pw_c128 *vg_dev, int *half_host);

/* Eigenmodes of every slice 0..N+1 at transverse wavevector kpar[2]
 * (Eq. loc / App. A Eq. A8): En_dev[(N+2)*N_G] ascending per slice and
 * U_dev[(N+2)*N_G*N_G], column j of slice q's block = eigenvector of E_n[j].
 * Either output may be NULL. */
pw_status pw_slice_modes(pw_ctx *ctx, const double *kpar, double *En_dev, pw_c128 *U_dev);

/* Interface overlaps O_p = U_p^H U_{p+1}, p = 0..N, i.e. the sums
 * sum_s (M^{p+1}_{js})^* M^p_{ns} of App. A Eq. transfer, at kpar[2]:
 * O_dev[(N+1)*N_G*N_G]. */
pw_status pw_overlaps(pw_ctx *ctx, const double *kpar, pw_c128 *O_dev);

/* Interface scattering matrix S(iface, iface+1), iface in 0..N, for npts
 * points (E[i], kpar[2i..2i+1]) (App. A Eqs. transfer and scatter):
 * S_dev[npts * 4 * N_G * N_G], per point the blocks S11, S12, S21, S22. */
pw_status pw_slice_smatrix(pw_ctx *ctx, int npts, const double *E, const double *kpar,
                           int iface, pw_c128 *S_dev);

/* Star product S(m,k) = S(m,n) * S(n,k) of Eq. recurrence for npts pairs of
 * caller-supplied scattering matrices (same layout as pw_slice_smatrix);
 * Sab_dev may not alias the inputs. */
pw_status pw_compose(pw_ctx *ctx, int npts, const pw_c128 *Sa_dev, const pw_c128 *Sb_dev,
                     pw_c128 *Sab_dev);

/* The mixed element of interface (iface, iface+1) for layer doubling with
 * App. A Eq. recurrence2: the transfer blocks I11 = P E-, I12 = Q E+ of
 * Eq. transfer and the scattering blocks S21, S22 of Eq. scatter (P, Q the
 * interface's matching blocks, E-+ = diag(e^{-+ik^{iface+1} dz})), for npts
 * points: T_dev[npts * 4 * N_G * N_G], per point the blocks I11, I12, S21,
 * S22 (column-major).  I11 carries the growing exponentials of evanescent
 * modes.  FP64.  Returns PW_ESINGULAR if an interface's P has a zero pivot. */
pw_status pw_slice_mixed(pw_ctx *ctx, int npts, const double *E, const double *kpar, int iface,
                         pw_c128 *T_dev);

/* One step of App. A Eq. recurrence2 (no nonlocal terms) for npts pairs of
 * mixed elements (layout of pw_slice_mixed): with X = I11(m,n) + I12(m,n) S21(n,k),
 *   I11(m,k) = X I11(n,k),  I12(m,k) = X I12(n,k) + I12(m,n) S22(n,k),
 *   S21(m,k) = S21(m,n) + S22(m,n) S21(n,k) X^-1,
 *   S22(m,k) = S22(m,n) S22(n,k) - S22(m,n) S21(n,k) X^-1 I12(m,n) S22(n,k).
 * Tab_dev may not alias the inputs.  FP64; PW_ESINGULAR on a zero pivot of X. */
pw_status pw_compose_mixed(pw_ctx *ctx, int npts, const pw_c128 *Ta_dev, const pw_c128 *Tb_dev,
                           pw_c128 *Tab_dev);

/* T(E, k_par) by layer doubling (App. A Eq. recurrence2, then Eq. recurrence):
 * for each point the N+1 interfaces' mixed elements are combined pairwise,
 * level by level (an odd last block moves up unchanged), with Eq. recurrence2
 * while the 1-norm of every block's I11 (largest absolute column sum) stays
 * at most cond_max; once one exceeds it (checked on the elements and after
 * each level), every block becomes its scattering matrix by Eq. scatter
 * (S11 = I11^-1, S12 = -I11^-1 I12) and the rest uses Eq. recurrence.  Then
 * t and T as in pw_transmission.  T_dev: device, npts doubles; levels_host:
 * NULL or npts ints, the mixed levels done per point (-1 at a threshold).
 * FP64 throughout (any precision of the context), one point after another,
 * synchronises the stream.  Device memory: the N+1 elements of a point and
 * half as many for the next level (64 N_G^2 bytes each), and work for up to
 * 2 x SMs combinations at a time (64 N_G^2 bytes each).
 * cond_max <= 0 or NaN: PW_EINVAL.  PW_ETHRESH (T = NaN there) and
 * PW_ESINGULAR as for pw_transmission.  A latency-oriented path (its
 * combinations run one CTA each); pw_transmission is the throughput path. */
pw_status pw_transmission_doubling(pw_ctx *ctx, int npts, const double *E, const double *kpar,
                                   double cond_max, double *T_dev, int *levels_host);

/* The forward hot path: for each point (E[i], kpar[2i..2i+1]) the junction's
 * S11(0,N+1) by a left-to-right sweep of star products over all N+1
 * interfaces, then t_ij = sqrt(k_i^R / k_j^L) S11_ij on open channels and
 * T = Tr(t^H t) (App. C, Sec. II B).
 *   T_dev[npts]                      transmission (required)
 *   t_dev[npts * N_G * N_G] or NULL  t, top-left n_open^R x n_open^L block of
 *                                    each N_G x N_G column-major slot
 *   nopen_dev[2 * npts] or NULL      (n_open^L, n_open^R) per point
 *   err_dev[npts] or NULL            estimated relative error of T: 0 for FP64;
 *                                    for PW_MIXED_FP32 the relative change of T
 *                                    made by the last refinement pass times the
 *                                    contraction c_i / c_{i-1} of the sizes of
 *                                    the last two corrections (the error left
 *                                    after that pass)
 * A point at an electrode threshold gets T = NaN and the call returns
 * PW_ETHRESH after finishing the others; a zero pivot gives PW_ESINGULAR,
 * and a tensor-core completion wait of the mixed form that ran out (bounded,
 * the kernel skips its result instead of hanging) gives PW_ETIMEOUT; both
 * latch in the context. */
pw_status pw_transmission(pw_ctx *ctx, int npts, const double *E, const double *kpar,
                          double *T_dev, pw_c128 *t_dev, int *nopen_dev, double *err_dev);

/* Adjoint: the weighted summed transmission  sumT = sum_i w_i T(E_i, kpar_i)
 * and its derivatives with respect to the depths v0 of the device-region
 * wells (pw_setup_desc.well_v0), computed in FP64 whatever the context's
 * precision.  For the slice model the constant Wronskian of a scattering
 * state c_j (incident from the left electrode) and a state d_i of the
 * transposed problem (incident from the right electrode) gives
 *   dt_ij = (1 / (2 i k_i^R)) sum_p int_{slice p} d_i^T (dH_p) c_j dz,
 * closed-form in each slice's modes (Eq. loc); both families of states come
 * from stored sweeps (Eqs. transfer, scatter, recurrence) and a backward pass.
 *   weight      host, npts, or NULL for w_i = 1
 *   sumT_host   host scalar (required)
 *   dV0_host    host, n_wells, or NULL (PW_EINVAL if the context was set up
 *               from explicit Fourier tables, which carry no wells)
 *   dgap_host   host scalar, or NULL: d sumT / d theta for the motion that
 *               pw_setup_desc.well_shift_rate / lead_shift_rate describe
 *               (PW_EINVAL if the context was set up with neither).  A well
 *               moved by delta changes its table by the factor e^{-i dG.delta}
 *               (a slice integral as above).  An electrode translated by delta
 *               has modes D U, D = diag(e^{-i G.delta}); expressed in the
 *               unmoved electrode's modes the scattering state jumps by
 *               (D^H - 1) c at the contact plane, so the Wronskian jumps there
 *               by -/+ i (d^T Gd c' - d'^T Gd c), Gd = diag(G.delta), minus at
 *               the left contact and plus at the right one; that jump takes
 *               the place of the slice integral.
 * The sweeps are recomputed in segments of C interfaces (pw_set_grad_checkpoint,
 * default C = ceil(sqrt(N+1))): a first pass keeps only the sweep state (the
 * accumulated S12 and the S11 columns) at the start of every segment; the
 * backward pass then takes the segments from the right, recomputing each
 * one's interfaces with their stores (Z_p, u_p) before stepping through it.
 * Synchronises the context's stream.  Device memory per point of a batch, in
 * complex doubles: (ceil((N+1)/C) - 1 + C)(n^2 + n n_c) for the checkpoints
 * and one segment's stores (about 2 sqrt(N+1) n^2), plus 4 (N+2) n n_c for
 * the amplitudes of both problems, plus the sweep's own n^2 + n (2n + n_c);
 * per call, 2 C n^2 for the gradient's slices, taken C at a time. */
pw_status pw_grad(pw_ctx *ctx, int npts, const double *E, const double *kpar, const double *weight,
                  double *sumT_host, double *dV0_host, double *dgap_host);

/* Separable nonlocal projector terms (Sec. II A, Eqs. kse0 / ksep: the term
 * sum_alpha C_alpha W_alpha(r) of the slice equation with
 * C_alpha = sum_beta D_alpha,beta <W_beta | psi>; Eqs. nloc / gsol_p0: each
 * slice's particular solutions; Eq. calm_0 for C; together the M X = D
 * system of App. C Eq. trans, without electrode-crossing projectors).  The
 * projectors are Bloch sums over the transverse cell of Gaussians
 * W_alpha(r) = exp(-|r - tau_alpha|^2 / 2 sigma_alpha^2) for
 * z_lo <= z <= z_hi (zero elsewhere; keep the range inside the device).
 *   m           number of projectors, 0..8 (0 removes them)
 *   params      host, 6 per projector: tau_x, tau_y, tau_z, sigma, z_lo, z_hi (bohr)
 *   D           host, m x m complex, row-major: D[alpha * m + beta]
 *   quad_nodes  Gauss-Legendre nodes per slice of the z integrals, 2..32
 * Synchronises the stream; PW_EINVAL for out-of-range arguments. */
pw_status pw_set_projectors(pw_ctx *ctx, int m, const double *params, const pw_c128 *D, int quad_nodes);

/* T(E, k_par) with the projector terms of pw_set_projectors, in FP64 whatever
 * the context's precision: psi = psi_0 + sum_alpha C_alpha psi_alpha (psi_0
 * the local scattering state, psi_alpha the response to projector alpha's
 * particular solutions with no incident wave) from one stored sweep whose
 * right-hand sides carry both, the backward pass for every slice's amplitudes,
 * then Eq. calm_0's m x m system per incident channel.
 *   T_dev   device, npts doubles (NaN for a threshold point or a singular system)
 *   C_dev   device or NULL: npts x m x N_G complex; C_alpha of incident left
 *           channel j at [i][alpha][j], j < n_open^L
 * PW_EINVAL when no projectors are set or the left electrode has more than 64
 * open channels; PW_ETHRESH and PW_ESINGULAR as for pw_transmission.
 * Synchronises the stream.  Memory per point as for pw_grad's one problem,
 * plus 4 (N+2) m N_G complex doubles. */
pw_status pw_transmission_nonlocal(pw_ctx *ctx, int npts, const double *E, const double *kpar, double *T_dev,
                                   pw_c128 *C_dev);

/* Segment length C of pw_grad's checkpointed recomputation: 0 (the default)
 * takes C = ceil(sqrt(N+1)); C >= N+1 stores every interface in one pass (no
 * recomputation).  PW_EINVAL for interval < 0.  The paper has no adjoint;
 * this is a memory/compute trade-off of pw_grad only (results are the same). */
pw_status pw_set_grad_checkpoint(pw_ctx *ctx, int interval);

/* Bytes of device memory the context's per-call workspaces hold now (the
 * buffers grown by pw_transmission, pw_grad and the mode stage; not the
 * per-k_par mode cache set up by pw_setup), into *bytes. */
pw_status pw_workspace_bytes(const pw_ctx *ctx, double *bytes);

/* Conductance sums of Sec. II B in FP64 on the device, for T of npts points
 * (as written by pw_transmission): out_dev[0] = sum_i w_i T_i (w_i = 1 when
 * weight_dev is NULL); out_dev[1] = Tbar of Eq. T1_d / T2_d, the mean of T_i
 * over the points at which the left electrode has an open channel
 * (nopen_dev[2i] > 0, the k_par mesh points of the electrode's conduction
 * channels; every point when nopen_dev is NULL), 0 when there is none;
 * out_dev[2] = that number of points.  Points with T = NaN (electrode
 * thresholds) are left out of both.  All pointers are device pointers;
 * asynchronous on cuda_stream (cudaStream_t, NULL = default); the summation
 * order is fixed, so the result is reproducible. */
pw_status pw_reduce_transmission(int npts, const double *T_dev, const int *nopen_dev, const double *weight_dev,
                                 double *out_dev, void *cuda_stream);

/* The star product of pw_compose for callers that must not allocate device
 * memory at all (no context, no cudaMalloc): for instance code running inside
 * a host application whose own memory manager owns the whole device, where a
 * cudaMalloc from a library would fail or fragment that pool, or code that
 * needs a fixed, known device-memory footprint.  The paper has no counterpart;
 * this is a deployment variant of pw_compose.
 *   n                N_G of the matrices (1 <= n <= 362)
 *   npts             number of (Sa, Sb) pairs
 *   Sa_dev, Sb_dev   device, npts x 4 blocks (S11, S12, S21, S22) of n x n
 *                    column-major complex, as for pw_compose
 *   Sab_dev          device output, same layout; may not alias the inputs
 *   cuda_stream      cudaStream_t on the current device (NULL = default)
 * Scratch: a fixed 8 MiB array inside the library's device image, held by
 * every GPU that loads the library until the process exits; batches larger
 * than the array run through it in chunks, and n above 362 (one point's
 * scratch would exceed 8 MiB) returns PW_EINVAL before any device work.  The
 * first call on each device looks up the array's device address (set-up
 * without allocation).  The call cannot be recorded into a CUDA graph: it
 * synchronises its stream before returning (it reads back the pivot status
 * of every launch), which a stream under capture does not allow.  All calls
 * share the one array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race; PW_ESINGULAR on a zero pivot. */
pw_status pw_compose_noalloc(int n, int npts, const pw_c128 *Sa_dev, const pw_c128 *Sb_dev,
                             pw_c128 *Sab_dev, void *cuda_stream);

/* FP64 kept for near-singular blocks in the mixed form (PW_MIXED_FP32;
 * Sec. II A's pivoted LU of the interface blocks, whose conditioning the
 * evanescent channels' wavenumbers set).  After a batch's FP32 sweep and
 * refinement, pw_transmission solves a point again with the FP64 sweep
 * (every interface in FP64; its T, t, n_open then come from that solve and
 * its error estimate is 0) when
 *   - the LU factors of some interface block W_p have a diagonal spread
 *     max|u_ii| / min|u_ii| above pivot_ratio_max (W_p's condition number is
 *     then at least that large), or
 *   - the refinement's estimated remaining error of the point is above
 *     err_max after its last pass, or
 *   - the FP32 sweep met a zero pivot.
 * Defaults 1e6 and 1e-8.  pivot_ratio_max < 0 turns the fallback off;
 * pivot_ratio_max = 0 sends every point to FP64.  PW_EINVAL for NaN or
 * err_max < 0.  Host setting, no device work. */
pw_status pw_set_fp64_fallback(pw_ctx *ctx, double pivot_ratio_max, double err_max);

/* Of the last pw_transmission call: *points = how many points the FP64
 * fallback solved again, *max_pivot_ratio = the largest diagonal spread of
 * any W_p's FP32 LU factors over its points (0 in the FP64 form). */
pw_status pw_get_fp64_fallback(const pw_ctx *ctx, int *points, double *max_pivot_ratio);

/* Launch variant of the star-product sweep of pw_transmission (default 2 for
 * PW_MIXED_FP32, 0 for PW_FP64).  The result is the same to the form's
 * accuracy for every variant; only the kernels differ.
 * Bit 0: 512-thread CTAs with 128 x 64 SIMT GEMM tiles (else 256 threads with
 * 64 x 64 tiles).  PW_MIXED_FP32 only: bit 1, the GEMM phases of every
 * interface ([W|Y], the LU's trailing updates, the triangular solves'
 * updates) on the fifth-generation tensor cores (tcgen05, TF32 operands split
 * into hi + lo parts, three products accumulated in FP32 in tensor memory),
 * with the LU's 32-column panels and the back substitution's 32-row blocks
 * taken in pairs so that the wide updates run with K = 64;
 * bit 2 (with bit 1), [W|Y] of point pairs in an FP16 split with row scales;
 * bit 3 (with bit 1), LAPACK-ordered pivots, the LU on W alone and the right-
 * hand sides eliminated in 128-row triangular blocks afterwards; bit 4, the
 * refinement's residual products as exact BF16 slice products on the tensor
 * cores (used when every point of a launch shares one k_par and N_G is a
 * multiple of 4 up to 512); bit 5, the slice eigenmodes and the overlaps in
 * double-float instead of FP64 (a mode stage about 4x faster, but 48-bit
 * modes: at a sharp antiresonance of T the error on T can exceed 1e-8
 * relative); bit 6, a batch of 32 points or more swept as two point groups
 * on two streams (the context's stream and a second one the context owns),
 * so that one group's latency-bound kernels run beside the other's wide
 * ones.  The mode cache of a k_par is kept across variant changes; set
 * the variant before the first call.  PW_EINVAL for a variant the context's
 * precision does not have (0..1 for PW_FP64, 0..127 for PW_MIXED_FP32). */
pw_status pw_set_sweep_variant(pw_ctx *ctx, int variant);

/* Timing of the library's own launches (for benchmarks and roofline
 * accounting).  While enabled, CUDA events on the context's stream bracket
 * every stage: the slice-mode stage (Hamiltonian assembly and eigensolver), the
 * overlap GEMMs, each batch of sweep launches, each batch's refinement, and
 * every [W|Y] GEMM launch of the sweep.  pw_get_profile synchronises the
 * stream and writes out[10] = {sweep ms, sweep launches, mode-stage ms, mode
 * stages, overlap ms, overlap stages, refinement ms, refinement passes,
 * [W|Y] GEMM ms, [W|Y] GEMM launches}; reset != 0 clears the records. */
pw_status pw_set_profiling(pw_ctx *ctx, int enable);
pw_status pw_get_profile(pw_ctx *ctx, double *out, int reset);

/* Per-kernel launch timing, gathered while profiling is on (enable >= 1 in
 * pw_set_profiling; enable = k brackets every k-th launch of each kernel kind
 * with CUDA events on the stream that kernel is launched on, and counts every
 * launch).  Kinds are numbered 0 .. pw_kernel_kinds()-1 and named by
 * pw_kernel_kind_name (a static string: the kernel, or the kernels that share
 * a role).  pw_get_kernel_profile synchronises the context's stream and
 * writes, for each kind k, out[3k] = summed ms of its timed launches,
 * out[3k+1] = its timed launches, out[3k+2] = all its launches; reset != 0
 * clears the counts.  Timing covers pw_transmission, pw_transmission_doubling
 * and pw_grad; the paper has no counterpart (measurement only). */
int pw_kernel_kinds(void);
const char *pw_kernel_kind_name(int kind);
pw_status pw_get_kernel_profile(pw_ctx *ctx, double *out, int reset);

/* Uneven batches: many independent problems, each with its own cell, basis
 * size N_G, slicing and potential, evaluated at one (E, k_par) point each.
 * The paper treats one junction at a time (Sec. II); a batch runs the same
 * steps for every instance (slice modes, overlaps, Eqs. transfer / scatter /
 * recurrence, App. C), with instances of equal N_G sharing launches: one
 * eigensolver launch over all their slices, and one sequence of sweep launches
 * over (tiles x instances) in which an instance with fewer slices drops out
 * after its last interface.
 *   n_inst        number of instances (>= 1)
 *   descs         host, n_inst problem descriptions as for pw_setup; every
 *                 description must use the same precision and refine_iters
 *   cuda_stream   as for pw_setup
 * On success *out owns the instances' geometry (one internal context each). */
pw_status pw_setup_batch(int n_inst, const pw_setup_desc *descs, void *cuda_stream, pw_batch **out);

/* T of instance i at (E[i], kpar[2i..2i+1]) into T_dev[i], for i < n_inst.
 *   E, kpar        host, n_inst and 2 n_inst values
 *   T_dev          device, n_inst doubles (required)
 *   nopen_dev      device, 2 n_inst ints (n_open^L, n_open^R), or NULL
 *   err_dev        device, n_inst doubles as for pw_transmission, or NULL
 * Instances are grouped by N_G (largest first) and each group is cut into
 * chunks that fit the free device memory.  Each chunk's sweep is recorded once
 * into a CUDA graph and replayed as one graph launch (pw_batch_set_options).
 * The sweep variant (pw_set_sweep_variant) is chosen per N_G by timing the
 * first interface steps of the group's first chunk with each variant (CUDA events),
 * and kept for the batch's later calls.  A threshold point gets T = NaN and the
 * call returns PW_ETHRESH after finishing the others; PW_ESINGULAR as for
 * pw_transmission.  Synchronises the stream. */
pw_status pw_transmission_batch(pw_batch *b, const double *E, const double *kpar, double *T_dev,
                                int *nopen_dev, double *err_dev);

/* Options of a batch: use_graph (1 = record and replay each chunk's sweep as a
 * CUDA graph, 0 = launch it directly), variant (-1 = autotune per N_G, else a
 * sweep variant as for pw_set_sweep_variant, for every size).  The mixed
 * form's eigenmodes and overlaps are FP64 unless a forced variant has bit 5
 * (double-float). */
pw_status pw_batch_set_options(pw_batch *b, int use_graph, int variant);

/* Stage times of the last pw_transmission_batch, out[8] = {slice-mode ms,
 * overlap ms, sweep ms, refinement ms, autotuning ms, chunks, graph launches,
 * sweep launches}, and the tile variant chosen per N_G: variants[i] for
 * ng[i], i < *n_sizes (at most max_sizes entries written). */
pw_status pw_batch_get_stats(const pw_batch *b, double *out, int *ng, int *variants, int max_sizes,
                             int *n_sizes);

void pw_batch_destroy(pw_batch *b);

/* Self-test of the tensor-core path used by the FP32 sweep: one 128 x 64
 * tile product with K = 32 on the fifth-generation tensor cores (tcgen05,
 * TF32 inputs, FP32 accumulation in tensor memory), compared on the host with
 * an FP64 product of the same FP32 inputs.  Writes the relative error
 * max|C - C_ref| / max|C_ref| of a single TF32 product (about 1e-3) and of
 * the three-product split A_hi B_hi + A_hi B_lo + A_lo B_hi (FP32 level,
 * about 1e-6).  Runs on the current device and synchronises it; returns
 * PW_ETIMEOUT if the tensor core did not signal completion within its bounded
 * wait.  The paper has no counterpart; this is a deployment check. */
pw_status pw_selftest_tensor_core(double *rel_err_tf32, double *rel_err_split);

/* Self-test of the exact-slice product behind the mixed form's residual when
 * every point shares its overlaps: O y as a sum of products of 7-bit slices
 * (BF16 on the tensor cores, FP32 accumulation that is exact for 2n <= 1024
 * inner terms, the slice pairs summed in double-float).  Runs that kernel on
 * random slices for a basis of n functions (a multiple of 4, at most 512) and
 * ncol columns (1..4096): first with only the leading slices non-zero and rows
 * and columns at full scale, where *mismatches counts the results that differ
 * from the exact integer product in any bit; then with every slice random,
 * where *rel_err = max|Y - Y_exact| / max|Y_exact| on every 64th row (about
 * 1e-14 expected).  Runs on the current device and synchronises it; returns
 * PW_EINVAL for sizes out of range and PW_ETIMEOUT if a tensor-core wait ran
 * out.  A deployment check with no counterpart in the paper. */
pw_status pw_selftest_slice_product(int n, int ncol, long long *mismatches, double *rel_err);

/* Self-test of the FP16 split used by sweep variant bit 2: the same 128 x 64
 * tile product with K = 32 as hi/lo FP16 parts (kind::f16, three MMAs per K
 * step of 16, operands scaled by the split's 2^8 headroom), against an FP64
 * product of the same FP32 inputs: *rel_err = max|C - C_ref| / max|C_ref|
 * (FP32 level, about 1e-7, expected).  Runs on the current device and
 * synchronises it; PW_ETIMEOUT if the tensor core did not signal completion
 * within its bounded wait.  A deployment check with no counterpart in the paper. */
pw_status pw_selftest_f16_split(double *rel_err);

/* Periodic electrodes (App. B, C; no nonlocal terms).  Each electrode is a
 * z-periodic cell of M slices (their Fourier tables in the layout of
 * pw_potential_tables, i.e. (2 Dm + 1) x (2 Dn + 1) values per slice with the
 * context's (Dm, Dn), in order along +z; thicknesses dz[M], bohr) whose third
 * lattice vector has the transverse part a3_perp[2] (0, 0 for a straight
 * cell; a tilted cell's next period is the present one moved by a3, so its
 * slice modes are D U with D = diag(e^{-i G.a3_perp})).  side 0: the left
 * electrode, whose last slice meets the device; side 1: the right electrode,
 * whose first slice meets the device.  Synchronises the stream. */
pw_status pw_set_periodic_electrode(pw_ctx *ctx, int side, int M, const pw_c128 *tables, const double *dz,
                                    const double *a3_perp);

/* T between the two periodic electrodes of pw_set_periodic_electrode, FP64
 * whatever the context's precision, for npts points (T_dev: device, npts
 * doubles).  Per electrode and point: the cell's S over one period (Eqs.
 * transfer, scatter, recurrence), its generalised Bloch states from Eq. cmp
 * (through the Cayley map mu = (lambda - s)/(lambda + s) to a bounded
 * standard eigenproblem, its complex Schur form and reordered invariant
 * subspaces: decaying for |lambda| < 1, growing for |lambda| > 1;
 * propagating states split by the sign of their z-flux and scaled to unit
 * flux); then S of [left reference slice, device slices, right reference
 * slice] and App. C's matching for the incident propagating states:
 * T = sum |t|^2.  The device slices are the context's (its z-invariant
 * electrodes are not used).  A point whose Bloch states fail (a band edge, a
 * Schur form that does not converge) gets T = NaN and the call returns
 * PW_ENOTCONV after the others.  Synchronises the stream. */
pw_status pw_transmission_periodic(pw_ctx *ctx, int npts, const double *E, const double *kpar, double *T_dev);

/* Self-test of the device eigen-kernels used for the Bloch states: the complex
 * Schur form A = Z T Z^H of one N x N complex matrix (host, column-major) by
 * Householder reduction and the shifted QR iteration, then with select != 0
 * the diagonal entries with negative real part moved first (*count of them).
 * T_host, Z_host: N x N outputs.  PW_ENOTCONV if the iteration did not
 * converge.  Synchronises the device; the paper has no counterpart. */
pw_status pw_selftest_schur(int N, const pw_c128 *A_host, pw_c128 *T_host, pw_c128 *Z_host, int select, int *count);

/* Self-test of the bounded device-side waits: one CTA holds tensor memory and
 * waits, at most `polls` polls of 64 ns, on an mbarrier that no tensor-core
 * operation will complete; with signal == 0 nobody arrives, so the wait runs
 * out and the call returns PW_ETIMEOUT (the CTA frees its tensor memory and
 * the context stays usable); with signal != 0 the CTA arrives first and the
 * call returns PW_OK.  PW_EINVAL for polls < 1.  Synchronises the device.
 * The paper has no counterpart; this checks the library's failure handling. */
pw_status pw_selftest_bounded_wait(int polls, int signal);

/* Measured arithmetic peaks of the current device, in TFLOP/s:
 * tflops[0] = FP64 FMA on the SIMT pipe (DFMA), tflops[1] = the warp-level FP64
 * MMA (mma.sync m8n8k4, the FP64 tensor path sm_103a offers), tflops[2] = FP32
 * FMA.  Each is timed with CUDA events over a few tens of milliseconds of
 * independent FMA (or MMA) chains on every SM.  Allocates a small output
 * buffer, synchronises the device; the paper has no counterpart (these are the
 * roofline denominators of the FP64 form and of the double-float kernels). */
pw_status pw_measure_peaks(double *tflops);

/* How many slice Hamiltonians of order n the FP64 eigensolver (Eq. loc, the
 * slice eigenproblem) works on at once on the current device: the CTAs of
 * one matrix each that fit on every SM together, times the SM count.  A mode
 * stage of more matrices than this runs in waves; its partial last wave runs
 * beside the overlaps (Eq. transfer's U_p^H U_{p+1}) of the slices already
 * done.  *matrices = 0 when the solver cannot run at order n.  PW_EINVAL for
 * n < 1 or a null pointer.  Host query; no device memory is touched. */
pw_status pw_eig_wave(int n, int *matrices);

#ifdef __cplusplus
}
#endif

#endif /* PW_H */
