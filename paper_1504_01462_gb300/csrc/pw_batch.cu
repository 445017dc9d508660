// Uneven batches (pw_setup_batch / pw_transmission_batch): many independent
// problems, each with its own basis size, slicing and potential, at one
// (E, k_par) point each.
//
// Instances of equal N_G share launches.  Their slice Hamiltonians are laid
// out back to back (instance j owns matrices mb_j .. mb_j + N_j + 1), so one
// eigensolver launch covers every slice of every instance of a chunk, and the
// sweep runs over (tiles x instances) with per-instance offsets into the
// eigenvalue, overlap, thickness and store arrays (PointDesc).  The interface
// loop runs to the largest N of the chunk; an instance leaves it after its own
// last interface.  Each chunk's sweep is recorded into a CUDA graph and
// replayed as one launch.  The GEMM tile variant of the sweep is chosen per
// N_G by timing a few interface steps of the first chunk with each variant.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "../../include/pw.h"
#include "pw_internal.h"

using pw::PointDesc;

namespace {

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct pw_batch {
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;        // private stream the sweep graphs are recorded on
  int precision = PW_FP64;
  int refine_iters = 0;
  int num_sms = 152;
  pw_status err = PW_OK;
  std::vector<pw_ctx *> inst;
  std::vector<pw::CtxView> view;
  bool use_graph = true;
  int force_variant = -1;                 // -1: autotune per N_G
  std::map<int, int> variant;             // chosen sweep variant per N_G
  double stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  Buf HU, V, En, stat, O, O32, O32t, O32lo, dz, pts, R, M, piv, KV, status;
  Buf rowexp;   // row scales of the FP16-split [W|Y] (sweep variant bit 2)
  Buf Zst, Ust, LUst, PIVst, Xa, Xb, Fr, Gr, carry, tmp, corr;
  Buf eigws;                              // workspace of the double-float eigensolver
};

namespace {

pw_status blatch(pw_batch *b, pw_status s) {
  if (b && b->err == PW_OK && s != PW_OK) b->err = s;
  return s;
}

// A failed runtime call is reported once: the runtime's last-error state is
// cleared so that it does not resurface in a later, unrelated call.
#define BCK(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      cudaGetLastError();                                                                          \
      return blatch(b, e_ == cudaErrorMemoryAllocation ? PW_ENOMEM : PW_ECUDA);                   \
    }                                                                                              \
  } while (0)

pw_status grow(pw_batch *b, Buf &x, size_t bytes) {
  if (x.bytes >= bytes) return PW_OK;
  if (x.p) cudaFree(x.p);
  x.p = nullptr;
  x.bytes = 0;
  if (cudaMalloc(&x.p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
    cudaGetLastError();
    return blatch(b, PW_ENOMEM);
  }
  x.bytes = std::max<size_t>(bytes, 256);
  return PW_OK;
}

size_t held(const pw_batch *b) {
  const Buf *all[] = {&b->HU, &b->V, &b->En, &b->stat, &b->O, &b->O32, &b->O32t, &b->O32lo, &b->dz, &b->pts, &b->R, &b->M, &b->piv,
                      &b->KV, &b->status, &b->Zst, &b->Ust, &b->LUst, &b->PIVst, &b->Xa, &b->Xb,
                      &b->Fr, &b->Gr, &b->carry, &b->tmp, &b->corr, &b->eigws, &b->rowexp};
  size_t s = 0;
  for (const Buf *x : all) s += x->bytes;
  return s;
}

// Device bytes one instance of a chunk needs (nc: the padded open-channel
// count assumed for the estimate).
size_t instance_bytes(int n, int N, int nc, int precision, bool refine) {
  const size_t nn = (size_t)n * n, esz = precision == PW_FP64 ? sizeof(zc) : sizeof(cc);
  size_t b = (size_t)(N + 2) * (2 * nn * sizeof(zc) + n * sizeof(double) + sizeof(int) + sizeof(double)) +
             (size_t)(N + 1) * nn * (sizeof(zc) + (precision == PW_MIXED_FP32 ? 3 * sizeof(cc) : 0));
  b += nn * esz + (size_t)n * (2 * n + nc) * esz + 3 * (size_t)n * esz + n * sizeof(int) + 256;
  if (precision == PW_MIXED_FP32) b += pw::heev_ws_bytes(n, N + 2);
  if (refine)
    b += (size_t)(N + 1) * (2 * nn + (size_t)n * nc) * sizeof(cc) + (size_t)(N + 1) * n * sizeof(int) +
         (size_t)(2 * (N + 2) + 2 * (N + 1) + 1) * n * nc * sizeof(zc) + 2 * (size_t)n * nc * sizeof(cc);
  return b;
}

int count_open(const double *En, int n, double E, bool *th) {
  int c = 0;
  for (int i = 0; i < n; ++i) {
    if (fabs(E - En[i]) < pw::kThresholdRy) *th = true;
    if (En[i] < E) ++c;
  }
  return c;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// One chunk: instances `ids` of basis size n.
pw_status run_chunk(pw_batch *b, const std::vector<int> &ids, int n, const double *E, const double *kpar,
                    double *T_dev, int *nopen_dev, double *err_dev, pw_status *result) {
  const cudaStream_t s = b->stream;
  const int m = (int)ids.size();
  const size_t nn = (size_t)n * n;
  const bool refine = b->precision == PW_MIXED_FP32 && b->refine_iters > 0;
  const size_t esz = b->precision == PW_FP64 ? sizeof(zc) : sizeof(cc);
  // back-to-back layout: slices (N+2 per instance) and interfaces (N+1)
  std::vector<long long> mb(m), ob(m);
  long long nmat = 0, nov = 0;
  int maxN = 0;
  for (int j = 0; j < m; ++j) {
    const pw::CtxView &v = b->view[ids[j]];
    mb[j] = nmat;
    ob[j] = nov;
    nmat += v.N + 2;
    nov += v.N + 1;
    maxN = std::max(maxN, v.N);
  }
  pw_status st;
  if ((st = grow(b, b->HU, (size_t)nmat * nn * sizeof(zc))) || (st = grow(b, b->V, (size_t)nmat * nn * sizeof(zc))) ||
      (st = grow(b, b->En, (size_t)nmat * n * sizeof(double))) ||
      (st = grow(b, b->stat, (size_t)nmat * sizeof(int))) || (st = grow(b, b->O, (size_t)nov * nn * sizeof(zc))) ||
      (st = grow(b, b->dz, (size_t)nmat * sizeof(double))))
    return st;
  const bool mixed = b->precision == PW_MIXED_FP32;
  // the mixed form's modes and overlaps in FP64, or, when every size is forced
  // to a variant with bit 5, in double-float
  const bool dfe = mixed && b->force_variant >= 0 && (b->force_variant & 32);
  if (mixed && ((st = grow(b, b->O32, (size_t)nov * nn * sizeof(cc))) ||
                (st = grow(b, b->O32t, (size_t)nov * nn * sizeof(cc))) ||
                (st = grow(b, b->O32lo, (size_t)nov * nn * sizeof(cc)))))
    return st;
  if (dfe && (st = grow(b, b->eigws, pw::heev_ws_bytes(n, (int)nmat)))) return st;
  zc *HU = (zc *)b->HU.p, *O = (zc *)b->O.p;
  double *En = (double *)b->En.p;
  std::vector<double> dzh((size_t)nmat);
  for (int j = 0; j < m; ++j) {
    const pw::CtxView &v = b->view[ids[j]];
    memcpy(dzh.data() + mb[j], v.dz, (v.N + 2) * sizeof(double));
  }
  BCK(cudaMemcpyAsync(b->dz.p, dzh.data(), nmat * sizeof(double), cudaMemcpyHostToDevice, s));
  cudaEvent_t ev[8];
  for (auto &e : ev) BCK(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t *e;
    ~EvGuard() {
      for (int i = 0; i < 8; ++i) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  // slice modes: Hamiltonians, one eigensolver launch, overlaps
  BCK(cudaEventRecord(ev[0], s));
  for (int j = 0; j < m; ++j) {
    const pw::CtxView &v = b->view[ids[j]];
    const int i = ids[j];
    pw::launch_assemble_h(HU + mb[j] * nn, v.tab, v.mn, v.G, kpar[2 * i], kpar[2 * i + 1], n, v.N + 2, v.Dm,
                          v.Dn, s);
  }
  pw::launch_eig(HU, (zc *)b->V.p, En, (int *)b->stat.p, n, (int)nmat, s, dfe, dfe ? b->eigws.p : nullptr,
                 dfe ? b->eigws.bytes : 0);
  BCK(cudaGetLastError());
  BCK(cudaEventRecord(ev[1], s));
  for (int j = 0; j < m; ++j)
    pw::launch_overlaps(HU + mb[j] * nn, O + ob[j] * nn, n, b->view[ids[j]].N + 2, 1, s, dfe);
  if (mixed) pw::launch_overlaps_fp32(O, (cc *)b->O32.p, (cc *)b->O32t.p, (cc *)b->O32lo.p, n, (int)nov, s);
  BCK(cudaGetLastError());
  BCK(cudaEventRecord(ev[2], s));
  // electrode eigenvalues -> open channels
  std::vector<int> stat((size_t)nmat);
  std::vector<double> EL((size_t)m * n), ER((size_t)m * n);
  BCK(cudaMemcpyAsync(stat.data(), b->stat.p, nmat * sizeof(int), cudaMemcpyDeviceToHost, s));
  for (int j = 0; j < m; ++j) {
    const int N = b->view[ids[j]].N;
    BCK(cudaMemcpyAsync(EL.data() + (size_t)j * n, En + mb[j] * n, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(ER.data() + (size_t)j * n, En + (mb[j] + N + 1) * n, n * sizeof(double),
                        cudaMemcpyDeviceToHost, s));
  }
  BCK(cudaStreamSynchronize(s));
  for (int v : stat)
    if (v < 0) return blatch(b, PW_ENOTCONV);
  std::vector<PointDesc> pd(m);
  int nc = 1;
  for (int j = 0; j < m; ++j) {
    const int i = ids[j];
    bool th = false;
    const int nL = count_open(EL.data() + (size_t)j * n, n, E[i], &th);
    const int nR = count_open(ER.data() + (size_t)j * n, n, E[i], &th);
    PointDesc d;
    d.E = E[i];
    d.kset = 0;
    d.nL = nL;
    d.nR = nR;
    d.out = i;
    d.skip = th ? 1 : 0;
    d.N = b->view[i].N;
    d.dz_off = (int)mb[j];
    d.en_off = mb[j];
    d.o_off = ob[j];
    d.st_off = ob[j];
    d.x_off = mb[j];
    pd[j] = d;
    if (th) *result = PW_ETHRESH;
    else nc = std::max(nc, nL);
  }
  nc = (nc + 3) & ~3;
  const int ncols = 2 * n + nc;
  const size_t vec = (size_t)m * n * nc;
  if ((st = grow(b, b->R, (size_t)m * nn * esz)) || (st = grow(b, b->M, (size_t)m * n * ncols * esz)) ||
      (st = grow(b, b->piv, (size_t)m * n * sizeof(int))) || (st = grow(b, b->KV, (size_t)m * 3 * n * esz)) ||
      (st = grow(b, b->pts, (size_t)m * sizeof(PointDesc))) || (st = grow(b, b->status, (size_t)m * sizeof(int))) ||
      (mixed && (st = grow(b, b->rowexp, (size_t)m * 2 * n * sizeof(int)))))
    return st;
  if (refine &&
      ((st = grow(b, b->Zst, (size_t)nov * nn * sizeof(cc))) || (st = grow(b, b->LUst, (size_t)nov * nn * sizeof(cc))) ||
       (st = grow(b, b->PIVst, (size_t)nov * n * sizeof(int))) ||
       (st = grow(b, b->Ust, (size_t)nov * n * nc * sizeof(cc))) ||
       (st = grow(b, b->Xa, (size_t)nmat * n * nc * sizeof(zc))) ||
       (st = grow(b, b->Xb, (size_t)nmat * n * nc * sizeof(zc))) ||
       (st = grow(b, b->Fr, (size_t)nov * n * nc * sizeof(zc))) ||
       (st = grow(b, b->Gr, (size_t)nov * n * nc * sizeof(zc))) || (st = grow(b, b->carry, vec * sizeof(zc))) ||
       (st = grow(b, b->corr, (size_t)2 * m * sizeof(double))) || (st = grow(b, b->tmp, 2 * vec * sizeof(cc)))))
    return st;
  BCK(cudaMemcpyAsync(b->pts.p, pd.data(), m * sizeof(PointDesc), cudaMemcpyHostToDevice, s));
  pw::SweepArgs a;
  memset(&a, 0, sizeof(a));
  a.pts = (const PointDesc *)b->pts.p;
  a.En = En;
  a.O = O;
  a.O32 = mixed ? (const cc *)b->O32.p : nullptr;
  a.O32t = mixed ? (const cc *)b->O32t.p : nullptr;
  a.dz = (const double *)b->dz.p;
  a.R = b->R.p;
  a.M = b->M.p;
  a.piv = (int *)b->piv.p;
  a.status = (int *)b->status.p;
  a.T = T_dev;
  a.t = nullptr;
  a.nopen = nopen_dev;
  a.err = err_dev;
  a.n = n;
  a.N = maxN;
  a.nc = nc;
  a.Zst = refine ? b->Zst.p : nullptr;
  a.Ust = refine ? b->Ust.p : nullptr;
  a.LUst = refine ? b->LUst.p : nullptr;
  a.PIVst = refine ? (int *)b->PIVst.p : nullptr;
  a.KV = b->KV.p;
  a.mirror = 0;
  a.wy_pairs = pw::points_pair_up(pd.data(), m);
  a.rowexp = mixed ? (int *)b->rowexp.p : nullptr;
  // tile variant: timed on the first interface steps of this chunk
  int var = b->force_variant;
  if (var < 0) {
    auto it = b->variant.find(n);
    if (it != b->variant.end()) var = it->second;
  }
  if (var < 0) {
    const int steps = std::min(maxN, 3) + 1;
    float best = 0.f;
    BCK(cudaEventRecord(ev[3], s));
    for (int cand : pw::sweep_variant_candidates(b->precision)) {
      BCK(pw::prepare_sweep_batched(n, b->precision, cand));
      BCK(cudaMemsetAsync(b->status.p, 0, m * sizeof(int), s));
      BCK(cudaEventRecord(ev[6], s));
      for (int p = 0; p < steps; ++p) BCK(pw::launch_sweep_batched(a, m, p, b->precision, s, nullptr, nullptr, cand));
      BCK(cudaEventRecord(ev[7], s));
      BCK(cudaEventSynchronize(ev[7]));
      const float ms = elapsed(ev[6], ev[7]);
      if (var < 0 || ms < best) {
        best = ms;
        var = cand;
      }
    }
    BCK(cudaEventRecord(ev[4], s));
    BCK(cudaEventSynchronize(ev[4]));
    b->stats[4] += elapsed(ev[3], ev[4]);
    b->variant[n] = var;
  }
  // the sweep, recorded into a graph and replayed (or launched directly)
  BCK(pw::prepare_sweep_batched(n, b->precision, var));
  BCK(cudaMemsetAsync(b->status.p, 0, m * sizeof(int), s));
  BCK(cudaEventRecord(ev[3], s));
  if (b->use_graph) {
    // recorded on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured), replayed on the caller's stream
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (!b->capture) BCK(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    BCK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    for (int p = 0; p <= maxN && ce == cudaSuccess; ++p)
      ce = pw::launch_sweep_batched(a, m, p, b->precision, b->capture, nullptr, nullptr, var);
    const cudaError_t ee = cudaStreamEndCapture(b->capture, &g);
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return blatch(b, PW_ECUDA);
    }
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return blatch(b, ie == cudaErrorMemoryAllocation ? PW_ENOMEM : PW_ECUDA);
    }
    const cudaError_t le = cudaGraphLaunch(ge, s);
    cudaGraphExecDestroy(ge);   // released once the launch completes
    BCK(le);
    b->stats[6] += 1;
  } else {
    for (int p = 0; p <= maxN; ++p) BCK(pw::launch_sweep_batched(a, m, p, b->precision, s, nullptr, nullptr, var));
  }
  b->stats[7] += (double)(maxN + 1) * pw::sweep_batched_launches(n, b->precision, var);
  BCK(cudaEventRecord(ev[4], s));
  if (refine) {
    pw::RefineArgs r;
    memset(&r, 0, sizeof(r));
    r.pts = a.pts;
    r.En = En;
    r.O = O;
    r.O32 = a.O32;
    r.O32lo = mixed ? (const cc *)b->O32lo.p : nullptr;
    r.dz = a.dz;
    r.Zst = (const cc *)b->Zst.p;
    r.Ust = (cc *)b->Ust.p;
    r.LUst = (const cc *)b->LUst.p;
    r.PIVst = (const int *)b->PIVst.p;
    r.M = (cc *)b->M.p;
    r.piv = a.piv;
    r.status = a.status;
    r.Xa = (zc *)b->Xa.p;
    r.Xb = (zc *)b->Xb.p;
    r.Fr = (zc *)b->Fr.p;
    r.Gr = (zc *)b->Gr.p;
    r.carry = (zc *)b->carry.p;
    r.tmp = (cc *)b->tmp.p;
    r.corr = (double *)b->corr.p;
    r.corr_prev = r.corr + m;
    r.T = T_dev;
    r.t = nullptr;
    r.nopen = nopen_dev;
    r.err = err_dev;
    r.n = n;
    r.N = maxN;
    r.nc = nc;
    r.x_slots = nmat;
    r.st_slots = nov;
    r.piv_order = pw::stored_piv_order(var);   // the stored factors' pivot order
    int passes = 0;
    BCK(pw::launch_refine(r, m, std::min(2, b->refine_iters), b->refine_iters, pw::kRefineTolRel, s, &passes));
  }
  BCK(cudaEventRecord(ev[5], s));
  std::vector<int> sth(m);
  BCK(cudaMemcpyAsync(sth.data(), b->status.p, m * sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  b->stats[0] += elapsed(ev[0], ev[1]);
  b->stats[1] += elapsed(ev[1], ev[2]);
  b->stats[2] += elapsed(ev[3], ev[4]);
  b->stats[3] += elapsed(ev[4], ev[5]);
  b->stats[5] += 1;
  for (int v : sth)
    if (v == 2) return blatch(b, PW_ETIMEOUT);   // a tensor-core wait ran out
  for (int v : sth)
    if (v) return blatch(b, PW_ESINGULAR);
  return PW_OK;
}

}  // namespace

extern "C" {

pw_status pw_setup_batch(int n_inst, const pw_setup_desc *descs, void *cuda_stream, pw_batch **out) {
  if (!out || n_inst < 1 || !descs) return PW_EINVAL;
  *out = nullptr;
  for (int i = 1; i < n_inst; ++i)
    if (descs[i].precision != descs[0].precision || descs[i].refine_iters != descs[0].refine_iters)
      return PW_EINVAL;
  pw_batch *b = new (std::nothrow) pw_batch();
  if (!b) return PW_ENOMEM;
  b->stream = (cudaStream_t)cuda_stream;
  for (int i = 0; i < n_inst; ++i) {
    pw_ctx *c = nullptr;
    const pw_status st = pw_setup(&descs[i], cuda_stream, &c);
    if (st != PW_OK) {
      pw_batch_destroy(b);
      return st;
    }
    b->inst.push_back(c);
    b->view.push_back(pw::ctx_view(c));
  }
  b->precision = b->view[0].precision;
  b->refine_iters = b->view[0].refine_iters;
  b->num_sms = b->view[0].num_sms;
  *out = b;
  return PW_OK;
}

pw_status pw_batch_set_options(pw_batch *b, int use_graph, int variant) {
  if (!b || variant < -1 || variant >= pw::sweep_variants(b->precision)) return PW_EINVAL;
  b->use_graph = use_graph != 0;
  b->force_variant = variant;
  return PW_OK;
}

pw_status pw_transmission_batch(pw_batch *b, const double *E, const double *kpar, double *T_dev,
                                int *nopen_dev, double *err_dev) {
  if (!b || !E || !kpar || !T_dev) return PW_EINVAL;
  if (b->err) return b->err;
  for (double &x : b->stats) x = 0.0;
  const bool refine = b->precision == PW_MIXED_FP32 && b->refine_iters > 0;
  // groups by N_G, largest first
  std::map<int, std::vector<int>, std::greater<int>> groups;
  for (int i = 0; i < (int)b->view.size(); ++i) groups[b->view[i].n].push_back(i);
  pw_status result = PW_OK;
  for (auto &g : groups) {
    const int n = g.first;
    std::vector<int> &ids = g.second;
    size_t free_b = 0, total_b = 0;
    BCK(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = (size_t)(0.8 * (double)(free_b + held(b)));
    const int nc_est = std::min(n, 64);
    size_t i0 = 0;
    while (i0 < ids.size()) {
      std::vector<int> chunk;
      size_t bytes = 0;
      const int cap = 3 * b->num_sms;
      while (i0 < ids.size() && (int)chunk.size() < cap) {
        const size_t need = instance_bytes(n, b->view[ids[i0]].N, nc_est, b->precision, refine);
        if (!chunk.empty() && bytes + need > budget) break;
        bytes += need;
        chunk.push_back(ids[i0++]);
      }
      const pw_status st = run_chunk(b, chunk, n, E, kpar, T_dev, nopen_dev, err_dev, &result);
      if (st != PW_OK) return st;
    }
  }
  return result;
}

pw_status pw_batch_get_stats(const pw_batch *b, double *out, int *ng, int *variants, int max_sizes,
                             int *n_sizes) {
  if (!b) return PW_EINVAL;
  if (out) memcpy(out, b->stats, sizeof(b->stats));
  int k = 0;
  for (auto &kv : b->variant) {
    if (k < max_sizes) {
      if (ng) ng[k] = kv.first;
      if (variants) variants[k] = kv.second;
    }
    ++k;
  }
  if (n_sizes) *n_sizes = k;
  return PW_OK;
}

void pw_batch_destroy(pw_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (pw_ctx *c : b->inst) pw_destroy(c);
  Buf *all[] = {&b->HU, &b->V, &b->En, &b->stat, &b->O, &b->O32, &b->O32t, &b->O32lo, &b->dz, &b->pts, &b->R, &b->M, &b->piv,
                &b->KV, &b->status, &b->Zst, &b->Ust, &b->LUst, &b->PIVst, &b->Xa, &b->Xb,
                &b->Fr, &b->Gr, &b->carry, &b->tmp, &b->corr, &b->eigws};
  for (Buf *x : all)
    if (x->p) cudaFree(x->p);
  delete b;
}

}  // extern "C"
