// CUDA part of libdpf: device copies of Y_bus, workspaces, launch
// configuration, the batched solve (Alg. 1 for every case) and the
// evaluation entry points (S_calc; loss + adjoint gradients).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dpf_internal.h"
#include "dpf_kernels.cuh"
#include "dpf_dc.cuh"

using namespace dpf;

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? DPF_E_OOM : DPF_E_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
  } while (0)

#define CKLAUNCH()                                                                            \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess)                                                                    \
      return fail(DPF_E_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                  \
  } while (0)

#define TRY(x)               \
  do {                       \
    int s_ = (x);            \
    if (s_ != DPF_OK) return s_; \
  } while (0)

namespace {

// Launch with programmatic stream serialisation when `pdl` (see pdl_wait /
// pdl_release in the kernels), else as a plain stream-ordered launch.
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                   Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <class T>
int dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? DPF_E_OOM : DPF_E_CUDA, "cudaMalloc(%zu bytes): %s",
                n * sizeof(T), cudaGetErrorString(e));
  }
  return DPF_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

template <class T>
int upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
  TRY(dalloc(dst, src.size()));
  if (!src.empty()) CK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return DPF_OK;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Y_bus upload
// ---------------------------------------------------------------------------
static void free_device(DeviceYbus& d) {
  dfree(d.ent32); dfree(d.row_ptr); dfree(d.prow_ptr); dfree(d.ppos); dfree(d.col); dfree(d.dcval); dfree(d.dcinv); dfree(d.val64); dfree(d.ebr); dfree(d.dpos);
  dfree(d.type); dfree(d.p64); dfree(d.q64); dfree(d.vmset); dfree(d.p32); dfree(d.q32);
  dfree(d.perm); dfree(d.iperm); dfree(d.br_f); dfree(d.br_t); dfree(d.br_r); dfree(d.br_x);
  dfree(d.br_bch); dfree(d.br_tap); dfree(d.br_itap); dfree(d.bridge);
  d.ready = false;
}

extern "C" int dpf_ybus_upload(dpf_ybus* y, void* stream) {
  clear_error();
  if (!y) return fail(DPF_E_INVALID, "dpf_ybus_upload: NULL handle");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceYbus& d = y->dev;
  if (d.ready) free_device(d);
  const int n = y->n, m = y->m, nnz = y->nnz;
  std::vector<int4> ent(nnz);
  std::vector<double2> v64(nnz);
  for (int p = 0; p < nnz; ++p) {
    const float re = (float)y->ival_re[p], im = (float)y->ival_im[p];
    int4 e;
    e.x = y->icol[p];
    memcpy(&e.y, &re, 4);
    memcpy(&e.z, &im, 4);
    e.w = 0;
    ent[p] = e;
    v64[p] = make_double2(y->ival_re[p], y->ival_im[p]);
  }
  std::vector<uint8_t> type(n);
  std::vector<double> p64(n), q64(n), vms(n);
  std::vector<float> p32(n), q32(n);
  for (int i = 0; i < n; ++i) {
    const int o = y->perm[i];
    type[i] = y->bus_type[o];
    p64[i] = y->p_spec[o];
    q64[i] = y->q_spec[o];
    vms[i] = y->vm_set[o];
    p32[i] = (float)p64[i];
    q32[i] = (float)q64[i];
  }
  std::vector<int32_t> bf(m), bt(m);
  std::vector<double> itap(m), bdc(m);
  for (int e = 0; e < m; ++e) {
    bf[e] = y->iperm[y->f_bus[e]];
    bt[e] = y->iperm[y->t_bus[e]];
    itap[e] = 1.0 / (y->tap[e] == 0.0 ? 1.0 : y->tap[e]);
    bdc[e] = itap[e] / y->x[e];  // DC susceptance 1 / (x tau)
  }
  // DC matrix B in the internal CSR: -b_l off the diagonal, sum of b_l on it
  std::vector<double> dcval(nnz, 0.0);
  for (int i = 0; i < n; ++i)
    for (int p = y->irow_ptr[i]; p < y->irow_ptr[i + 1]; ++p) {
      const int l = y->iebr[p];
      if (l < 0) continue;
      dcval[p] = -bdc[l];
      dcval[y->idpos[i]] += bdc[l];
    }
  // as double-float pairs (hi, lo) for the DC solver
  auto pair = [](double v) {
    const float hi = (float)v;
    float2 r;
    r.x = hi;
    r.y = (float)(v - (double)hi);
    return r;
  };
  std::vector<float2> dcval2(nnz), dcinv2(n);
  for (int p = 0; p < nnz; ++p) dcval2[p] = pair(dcval[p]);
  for (int i = 0; i < n; ++i) {
    const double dii = dcval[y->idpos[i]];
    dcinv2[i] = pair(dii != 0.0 ? 1.0 / dii : 0.0);
  }
  int rc = DPF_OK;
  do {
    if ((rc = upload(&d.ent32, ent, s))) break;
    if ((rc = upload(&d.row_ptr, y->irow_ptr, s))) break;
    if ((rc = upload(&d.prow_ptr, y->iprow_ptr, s))) break;
    if ((rc = upload(&d.ppos, y->ippos, s))) break;
    if ((rc = upload(&d.col, y->icol, s))) break;
    if ((rc = upload(&d.val64, v64, s))) break;
    if ((rc = upload(&d.dcval, dcval2, s))) break;
    if ((rc = upload(&d.dcinv, dcinv2, s))) break;
    if ((rc = upload(&d.ebr, y->iebr, s))) break;
    if ((rc = upload(&d.dpos, y->idpos, s))) break;
    if ((rc = upload(&d.type, type, s))) break;
    if ((rc = upload(&d.p64, p64, s))) break;
    if ((rc = upload(&d.q64, q64, s))) break;
    if ((rc = upload(&d.vmset, vms, s))) break;
    if ((rc = upload(&d.p32, p32, s))) break;
    if ((rc = upload(&d.q32, q32, s))) break;
    if ((rc = upload(&d.perm, y->perm, s))) break;
    if ((rc = upload(&d.iperm, y->iperm, s))) break;
    if ((rc = upload(&d.br_f, bf, s))) break;
    if ((rc = upload(&d.br_t, bt, s))) break;
    if ((rc = upload(&d.br_r, y->r, s))) break;
    if ((rc = upload(&d.br_x, y->x, s))) break;
    if ((rc = upload(&d.br_bch, y->b_ch, s))) break;
    if ((rc = upload(&d.br_tap, y->tap, s))) break;
    if ((rc = upload(&d.br_itap, itap, s))) break;
    if ((rc = upload(&d.bridge, y->bridge, s))) break;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = fail(DPF_E_CUDA, "upload sync: %s", cudaGetErrorString(e)); break; }
  } while (0);
  if (rc != DPF_OK) {
    free_device(d);
    return rc;
  }
  cudaGetDevice(&d.device);
  d.ready = true;
  return DPF_OK;
}

extern "C" int dpf_build_ybus(const dpf_grid* g, void* stream, dpf_ybus** out) {
  if (!out) return fail(DPF_E_INVALID, "dpf_build_ybus: NULL out");
  *out = nullptr;
  dpf_ybus* y = nullptr;
  TRY(dpf_build_ybus_host(g, &y));
  const int rc = dpf_ybus_upload(y, stream);
  if (rc != DPF_OK) {
    delete y;
    return rc;
  }
  *out = y;
  return DPF_OK;
}

extern "C" int dpf_ybus_free(dpf_ybus* y) {
  if (!y) return DPF_OK;
  if (y->dev.ready) free_device(y->dev);
  delete y;
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
struct dpf_workspace {
  const dpf_ybus* y = nullptr;
  size_t cap_elems = 0;   // N * Kp capacity
  int cap_cases = 0;      // Kp capacity
  size_t cap_stage = 0;   // K * N capacity of the user-layout staging buffers
  // element buffers (sized for FP64; FP32 mode uses the front half)
  void *V = nullptr, *W = nullptr, *G0 = nullptr;
  void* ms = nullptr;  // master (theta, |V|) pairs, 16 bytes per element
  void* os = nullptr;  // optimiser moments, 4 values per element
  void *p = nullptr, *q = nullptr;
  double *p64 = nullptr, *q64 = nullptr, *tmp_a = nullptr, *tmp_b = nullptr, *tmp_c = nullptr;
  double2* V64 = nullptr;
  void *sbuf = nullptr, *cbuf = nullptr;
  // Y values rebuilt from caller branch parameters
  int4* ent_loc = nullptr;
  double2* val_loc = nullptr;
  // per-case buffers
  int32_t *active = nullptr, *iters = nullptr, *status = nullptr, *of = nullptr, *ot = nullptr;
  int32_t *bad = nullptr, *cool = nullptr;
  double *lr = nullptr, *best = nullptr, *out_max = nullptr, *out_loss = nullptr, *loss64 = nullptr;
  void *step_size = nullptr, *isbc2 = nullptr, *yff = nullptr, *yft = nullptr, *ytt = nullptr;
  double2 *yff64 = nullptr, *yft64 = nullptr, *ytt64 = nullptr;
  double *b1t = nullptr, *b2t = nullptr;
  int32_t* cand = nullptr;
  unsigned int* mx32 = nullptr;
  unsigned long long* maxmis = nullptr;
  int32_t* outage_dev = nullptr;
  int32_t* n_active = nullptr;
  int32_t* h_n_active = nullptr;  // pinned
  unsigned int* tile_cnt = nullptr;  // per case tile, for the forward pass's scheduler
  void* loss_part = nullptr;         // [row blocks][Kp] the forward pass's loss partials (8 B each)
  size_t cap_part = 0;
  double* dcs = nullptr;     // DC solver, per case: rz, rz', pq, rr, rr0, beta, res, b_out, flow ([9][Kp])
  int32_t* dci = nullptr;    // DC solver, per case: active, iters ([2][Kp]), then its active count
  int32_t* h_dc_nact = nullptr;  // pinned
  int cap_tiles = 0;
  int tiles = 0;  // case tiles of the scheduler (tile_cnt holds their counters first)
  // user-layout staging for host_io
  double *st_a = nullptr, *st_b = nullptr, *st_c = nullptr;
  cudaStream_t cap_stream = nullptr;
  // solve state
  bool begun = false;
  int K = 0, Kp = 0, lanes = 1, warps = 8, gx = 1, gy = 1, rpb = 1, smem = 0, precision = DPF_FP32;
  int gy_b = 1, rpb_b = 1, ysmem_b = 0;  // the adjoint pass's row blocks (may differ from the forward's)
  bool pairs = false;   // FP32 solve loop, Kp a multiple of 64: two cases per thread possible
  // shared-memory windows of V for the forward pass: per row block the first
  // and last row referenced (host copy + device copy)
  std::vector<int32_t> h_wlo, h_whi;
  int32_t *d_wlo = nullptr, *d_whi = nullptr;
  int cap_wblocks = 0;
  bool staged = false;
  int ysmem = 0;
  bool pair_fwd = false, pair_adj = false;
  bool direct = false;    // single-case FP32 solve: Y rows read from global memory (no staging)
  int4* pent = nullptr;   // padded Y entries of the direct view
  size_t cap_pent = 0;
  bool pid_ready = false;  // operating points staged by dpf_paramid_begin
  std::vector<std::pair<std::vector<long long>, std::vector<int>>> tune_cache;  // key -> (lanes, warps, rb, pairs)
  bool spec_per_case = false, has_outage = false;
  dpf_solve_opts opts;
  int t_done = 0;
  cudaGraphExec_t gexec = nullptr;
  int graph_kernels = 0;  // kernel nodes per replay
  bool use_local_y = false;
  long long launches = 0;
  // per-kernel timing
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_fwd, ev_adj;  // (start, stop) indices into ev_pool
  size_t ev_used = 0;
};

static void ws_free_buffers(dpf_workspace* w) {
  void** ptrs[] = {&w->V, &w->W, &w->G0, &w->ms, &w->os, &w->p, &w->q,
                   &w->sbuf, &w->cbuf, &w->step_size, &w->isbc2, &w->yff, &w->yft, &w->ytt};
  for (void** p : ptrs) dfree(*p);
  dfree(w->p64); dfree(w->q64); dfree(w->tmp_a); dfree(w->tmp_b); dfree(w->tmp_c); dfree(w->V64);
  dfree(w->ent_loc); dfree(w->val_loc);
  dfree(w->active); dfree(w->iters); dfree(w->status); dfree(w->of); dfree(w->ot); dfree(w->bad); dfree(w->cool);
  dfree(w->lr); dfree(w->best); dfree(w->out_max); dfree(w->out_loss); dfree(w->loss64);
  dfree(w->yff64); dfree(w->yft64); dfree(w->ytt64); dfree(w->maxmis); dfree(w->outage_dev);
  dfree(w->b1t); dfree(w->b2t); dfree(w->cand); dfree(w->mx32);
  dfree(w->dcs); dfree(w->dci);
  dfree(w->st_a); dfree(w->st_b); dfree(w->st_c);
  dfree(w->d_wlo); dfree(w->d_whi);
  dfree(w->pent);
  w->cap_pent = 0;
  w->cap_wblocks = 0;
  dfree(w->tile_cnt);
  w->cap_tiles = 0;
  dfree(w->loss_part);
  w->cap_part = 0;
  w->cap_elems = 0;
  w->cap_cases = 0;
  w->cap_stage = 0;
}

static void ws_drop_graph(dpf_workspace* w) {
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  w->gexec = nullptr;
  w->graph_kernels = 0;
}

static int ev_take(dpf_workspace* w, cudaEvent_t* e) {
  if (w->ev_used == w->ev_pool.size()) {
    cudaEvent_t n;
    CK(cudaEventCreate(&n));
    w->ev_pool.push_back(n);
  }
  *e = w->ev_pool[w->ev_used++];
  return DPF_OK;
}

// Grow the buffers to hold Kp cases (N * Kp elements) and K*N staging.
static int ws_reserve(dpf_workspace* w, int Kp, size_t stage) {
  const dpf_ybus* y = w->y;
  const size_t E = (size_t)y->n * Kp;
  if (E > w->cap_elems || Kp > w->cap_cases) {
    ws_drop_graph(w);
    dfree(w->V); dfree(w->W); dfree(w->G0); dfree(w->ms); dfree(w->os);
    dfree(w->p); dfree(w->q); dfree(w->sbuf); dfree(w->cbuf);
    dfree(w->p64); dfree(w->q64); dfree(w->tmp_a); dfree(w->tmp_b); dfree(w->tmp_c); dfree(w->V64);
    dfree(w->step_size); dfree(w->isbc2); dfree(w->yff); dfree(w->yft); dfree(w->ytt);
    dfree(w->active); dfree(w->iters); dfree(w->status); dfree(w->of); dfree(w->ot); dfree(w->bad);
    dfree(w->cool); dfree(w->lr); dfree(w->best); dfree(w->out_max); dfree(w->out_loss); dfree(w->loss64);
    dfree(w->yff64); dfree(w->yft64); dfree(w->ytt64); dfree(w->maxmis); dfree(w->outage_dev);
    dfree(w->b1t); dfree(w->b2t); dfree(w->cand); dfree(w->mx32);
    dfree(w->dcs); dfree(w->dci);
    w->cap_elems = 0;
    w->cap_cases = 0;
    char** bufs16[] = {(char**)&w->V, (char**)&w->W, (char**)&w->G0, (char**)&w->V64, (char**)&w->sbuf,
                       (char**)&w->cbuf, (char**)&w->ms};
    for (char** b : bufs16) TRY(dalloc(b, E * 16));
    TRY(dalloc((char**)&w->os, E * 32));
    char** bufs8[] = {(char**)&w->p, (char**)&w->q, (char**)&w->p64, (char**)&w->q64,
                      (char**)&w->tmp_a, (char**)&w->tmp_b, (char**)&w->tmp_c};
    for (char** b : bufs8) TRY(dalloc(b, E * 8));
    TRY(dalloc((char**)&w->step_size, (size_t)Kp * 8));
    TRY(dalloc((char**)&w->isbc2, (size_t)Kp * 8));
    TRY(dalloc((char**)&w->yff, (size_t)Kp * 16));
    TRY(dalloc((char**)&w->yft, (size_t)Kp * 16));
    TRY(dalloc((char**)&w->ytt, (size_t)Kp * 16));
    TRY(dalloc(&w->active, Kp)); TRY(dalloc(&w->iters, Kp)); TRY(dalloc(&w->status, Kp));
    TRY(dalloc(&w->of, Kp)); TRY(dalloc(&w->ot, Kp)); TRY(dalloc(&w->bad, Kp)); TRY(dalloc(&w->cool, Kp));
    TRY(dalloc(&w->lr, Kp)); TRY(dalloc(&w->best, Kp)); TRY(dalloc(&w->out_max, Kp));
    TRY(dalloc(&w->out_loss, Kp)); TRY(dalloc(&w->loss64, Kp));
    TRY(dalloc(&w->yff64, Kp)); TRY(dalloc(&w->yft64, Kp)); TRY(dalloc(&w->ytt64, Kp));
    TRY(dalloc(&w->maxmis, Kp)); TRY(dalloc(&w->outage_dev, Kp));
    TRY(dalloc(&w->b1t, Kp)); TRY(dalloc(&w->b2t, Kp)); TRY(dalloc(&w->cand, Kp)); TRY(dalloc(&w->mx32, Kp));
    TRY(dalloc(&w->dcs, (size_t)9 * Kp)); TRY(dalloc(&w->dci, (size_t)2 * Kp + 1));
    CK(cudaMemset(w->p64, 0, E * 8));
    CK(cudaMemset(w->q64, 0, E * 8));
    w->cap_elems = E;
    w->cap_cases = Kp;
  }
  if (stage > w->cap_stage) {
    dfree(w->st_a); dfree(w->st_b); dfree(w->st_c);
    w->cap_stage = 0;
    TRY(dalloc(&w->st_a, stage));
    TRY(dalloc(&w->st_b, stage));
    TRY(dalloc(&w->st_c, stage));
    w->cap_stage = stage;
  }
  if (!w->ent_loc && y->nnz > 0) {
    TRY(dalloc(&w->ent_loc, y->nnz));
    TRY(dalloc(&w->val_loc, y->nnz));
  }
  return DPF_OK;
}

extern "C" int dpf_workspace_create(const dpf_ybus* y, int32_t max_case, dpf_workspace** out) {
  clear_error();
  if (!y || !out) return fail(DPF_E_INVALID, "dpf_workspace_create: NULL argument");
  if (!y->dev.ready) return fail(DPF_E_STATE, "Y_bus is not on the device (dpf_ybus_upload)");
  if (max_case < 1) return fail(DPF_E_INVALID, "max_case must be >= 1");
  dpf_workspace* w = new (std::nothrow) dpf_workspace();
  if (!w) return fail(DPF_E_OOM, "out of host memory");
  w->y = y;
  dpf_default_opts(&w->opts);
  int rc = DPF_OK;
  do {
    if ((rc = dalloc(&w->n_active, 1))) break;
    cudaError_t e = cudaMallocHost((void**)&w->h_n_active, sizeof(int32_t));
    if (e != cudaSuccess) { rc = fail(DPF_E_OOM, "cudaMallocHost: %s", cudaGetErrorString(e)); break; }
    e = cudaMallocHost((void**)&w->h_dc_nact, sizeof(int32_t));
    if (e != cudaSuccess) { rc = fail(DPF_E_OOM, "cudaMallocHost: %s", cudaGetErrorString(e)); break; }
    e = cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { rc = fail(DPF_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); break; }
    const int Kp = max_case <= 16 ? pow2ceil(max_case) : (max_case + 31) / 32 * 32;
    if ((rc = ws_reserve(w, Kp, 0))) break;
  } while (0);
  if (rc != DPF_OK) {
    dpf_workspace_free(w);
    return rc;
  }
  *out = w;
  return DPF_OK;
}

extern "C" int dpf_workspace_free(dpf_workspace* w) {
  if (!w) return DPF_OK;
  ws_drop_graph(w);
  for (auto e : w->ev_pool) cudaEventDestroy(e);
  w->ev_pool.clear();
  ws_free_buffers(w);
  dfree(w->n_active);
  if (w->h_n_active) cudaFreeHost(w->h_n_active);
  if (w->h_dc_nact) cudaFreeHost(w->h_dc_nact);
  if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
  delete w;
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// Launch plumbing, one instance per precision
// ---------------------------------------------------------------------------
template <class R>
struct Plan {
  using C = typename Prec<R>::C;
  using M = typename Prec<R>::M;
  IterArgs<R> it;
  Check64Args<M> ck;
  ApplyArgs ap;
  dim3 grid, block;   // one case per thread
  dim3 cgrid;         // (the same; check and evaluation kernels)
  dim3 pgrid;         // two cases per thread
  IterArgs<R> itb;    // the adjoint pass (its own row blocks)
  dim3 gridb, pgridb;
  int smem;
  int ysmem;
  bool need_volt64;
};

template <class R>
static Plan<R> make_plan(dpf_workspace* w) {
  using C = typename Prec<R>::C;
  using M = typename Prec<R>::M;
  const dpf_ybus* y = w->y;
  const DeviceYbus& d = y->dev;
  Plan<R> P;
  memset(&P.it, 0, sizeof(P.it));
  memset(&P.ck, 0, sizeof(P.ck));
  memset(&P.ap, 0, sizeof(P.ap));
  IterArgs<R>& a = P.it;
  a.N = y->n;
  a.Kp = w->Kp;
  a.lanes = w->lanes;
  a.rpb = w->rpb;
  a.wlo = w->staged ? w->d_wlo : nullptr;
  a.whi = w->staged ? w->d_whi : nullptr;
  a.ysmem = w->ysmem;
  // FP32 iterations gate the FP64 test with the forward pass's FP32 mismatch
  const bool gated = (sizeof(R) == 4) && w->opts.gate > 0.0;
  a.prp = d.prow_ptr;
  a.ppos = d.ppos;
  a.pent = w->pent;
  const int4* ent = w->use_local_y ? w->ent_loc : d.ent32;
  const double2* v64 = w->use_local_y ? w->val_loc : d.val64;
  if constexpr (sizeof(R) == 4) {
    a.Y.ent = ent;
  } else {
    a.Y.col = d.col;
    a.Y.val = v64;
  }
  a.type = d.type;
  a.V = (C*)w->V;
  a.W = (C*)w->W;
  a.qpv = (R*)w->G0;  // the buffer holds Q_calc at pv buses
  a.ms = (typename Prec<R>::MS*)w->ms;
  a.os = (Mom<R>*)w->os;
  a.spec_per_case = w->spec_per_case ? 1 : 0;
  if (w->spec_per_case) {
    a.pspec = (const R*)w->p;
    a.qspec = (const R*)w->q;
  } else if constexpr (sizeof(R) == 4) {
    a.pspec = (const R*)d.p32;
    a.qspec = (const R*)d.q32;
  } else {
    a.pspec = (const R*)d.p64;
    a.qspec = (const R*)d.q64;
  }
  a.active = w->active;
  a.of = w->of;
  a.ot = w->ot;
  a.yff = (const C*)w->yff;
  a.yft = (const C*)w->yft;
  a.ytt = (const C*)w->ytt;
  a.has_outage = w->has_outage ? 1 : 0;
  a.loss_part = (R*)w->loss_part;
  a.mx32 = gated ? w->mx32 : nullptr;
  a.step_size = (const R*)w->step_size;
  a.isbc2 = (const R*)w->isbc2;
  a.beta1 = (R)w->opts.beta1;
  a.beta2 = (R)w->opts.beta2;
  a.eps = (R)w->opts.eps;
  a.inv_m2 = (R)(y->m_loss > 0 ? 2.0 / y->m_loss : 0.0);
  a.opt = w->opts.optimizer;
  a.mom = (R)w->opts.momentum;
  a.alpha = (R)w->opts.alpha;
  a.m_half = (R)(0.5 * y->m_loss);
  a.n_active = w->n_active;
  if constexpr (sizeof(R) == 4) {
    if (w->precision == DPF_FP32R) {  // references of the refined iterations (solve-loop buffers)
      a.vref = (const float2*)w->cbuf;
      a.irf = (const float4*)w->sbuf;
    }
    if (w->precision == DPF_MIXED) {
      a.V64m = (double2*)w->V;
      a.Y64.col = d.col;
      a.Y64.val = v64;
      a.pspec64 = w->spec_per_case ? w->p64 : d.p64;
      a.qspec64 = w->spec_per_case ? w->q64 : d.q64;
      a.yff64 = w->yff64;
      a.yft64 = w->yft64;
      a.ytt64 = w->ytt64;
      a.inv_m2_64 = y->m_loss > 0 ? 2.0 / y->m_loss : 0.0;
    }
  }

  SchedArgs<R>& s = a.sc;
  s.Kp = w->Kp;
  s.active = w->active;
  s.iters = w->iters;
  s.status = w->status;
  s.loss_part = (const R*)w->loss_part;
  s.grp_part = (R*)w->loss_part + (size_t)w->gy * w->Kp;
  s.grp_cnt = w->tile_cnt + w->tiles;
  s.mx32 = gated ? w->mx32 : nullptr;
  s.cand = w->cand;
  s.gate = w->opts.gate;
  s.b1t = w->b1t;
  s.b2t = w->b2t;
  s.lr = w->lr;
  s.best = w->best;
  s.bad = w->bad;
  s.cool = w->cool;
  s.step_size = (R*)w->step_size;
  s.isbc2 = (R*)w->isbc2;
  s.n_active = w->n_active;
  s.inv_m = y->m_loss > 0 ? 1.0 / y->m_loss : 0.0;
  s.beta1 = w->opts.beta1;
  s.beta2 = w->opts.beta2;
  s.factor = w->opts.factor;
  s.threshold = w->opts.threshold;
  s.min_lr = w->opts.min_lr;
  s.gamma = w->opts.gamma;
  s.lr0 = w->opts.lr;
  s.sched = w->opts.sched;
  s.patience = w->opts.patience;
  s.cooldown = w->opts.cooldown;
  s.step_every = std::max(1, w->opts.step_size);
  s.opt = w->opts.optimizer;

  a.tile_cnt = w->tile_cnt;  // NULL in the evaluation entry points: no scheduler there
  Check64Args<M>& c = P.ck;
  c.N = y->n;
  c.Kp = w->Kp;
  c.lanes = w->lanes;
  c.all_cases = 0;
  c.rp = d.row_ptr;
  c.col = d.col;
  c.val = v64;
  c.type = d.type;
  c.ms = (const typename Prec<R>::MS*)w->ms;
  P.need_volt64 = (sizeof(R) == 4);
  c.V64 = P.need_volt64 ? w->V64 : (double2*)w->V;
  c.pspec = w->spec_per_case ? w->p64 : d.p64;
  c.qspec = w->spec_per_case ? w->q64 : d.q64;
  c.spec_per_case = w->spec_per_case ? 1 : 0;
  c.active = w->active;
  c.cand = gated ? w->cand : nullptr;
  c.iters = w->iters;
  // refined FP32: the test at every 100th step (or every test, with longer
  // intervals) also re-anchors the cases the gate keeps out
  const int ce = std::max(1, w->opts.check_every);
  const int re = w->opts.refresh_every > 0 ? w->opts.refresh_every : 100;
  c.full_every = (gated && w->precision == DPF_FP32R) ? std::max(ce, re / ce * ce) : 0;
  c.of = w->of;
  c.ot = w->ot;
  c.yff = w->yff64;
  c.yft = w->yft64;
  c.ytt = w->ytt64;
  c.has_outage = w->has_outage ? 1 : 0;
  c.maxmis = w->maxmis;
  c.loss64 = w->loss64;
  c.n_active = w->n_active;
  c.refresh = 0;
  if (sizeof(R) == 4 && w->precision == DPF_FP32R) {
    c.vref = (float2*)w->cbuf;
    c.irf = (float4*)w->sbuf;
    c.dv = (float2*)w->V;
  }

  ApplyArgs& p = P.ap;
  p.K = w->K;
  p.Kp = w->Kp;
  p.final_pass = 0;
  p.tol = w->opts.tol;
  p.inv_m = y->m_loss > 0 ? 1.0 / y->m_loss : 0.0;
  p.active = w->active;
  p.cand = gated ? w->cand : nullptr;
  p.iters = w->iters;
  p.full_every = c.full_every;
  p.status = w->status;
  p.maxmis = w->maxmis;
  p.loss64 = w->loss64;
  p.out_max = w->out_max;
  p.out_loss = w->out_loss;
  p.n_active = w->n_active;

  P.cgrid = dim3(w->Kp / w->lanes, w->gy);
  P.grid = P.cgrid;
  P.pgrid = dim3(w->Kp / 64, w->gy);
  P.itb = P.it;
  P.itb.tile_cnt = nullptr;  // the scheduler runs in the forward pass only
  P.itb.rpb = w->rpb_b;
  P.itb.wlo = nullptr;
  P.itb.whi = nullptr;
  P.gridb = dim3(w->Kp / w->lanes, w->gy_b);
  P.pgridb = dim3(w->Kp / 64, w->gy_b);
  P.block = dim3(w->warps * 32);
  P.smem = w->smem;      // forward pass: Y rows + (optional) V window
  P.ysmem = w->ysmem_b;  // adjoint pass: its Y rows only
  return P;
}

template <class R>
static int launch_check(dpf_workspace* w, cudaStream_t s, bool final_pass) {
  Plan<R> P = make_plan<R>(w);
  P.ck.all_cases = final_pass ? 1 : 0;
  P.ck.refresh = (w->precision == DPF_FP32R && !final_pass) ? 1 : 0;
  P.ap.final_pass = final_pass ? 1 : 0;
  using M = typename Prec<R>::M;
  const bool pdl = w->opts.pdl != 0;
  if (P.need_volt64) {
    CK(launch(k_volt64<M>, P.cgrid, P.block, 0, s, pdl, P.ck));
    w->launches++;
  }
  CK(launch(k_check64<M>, P.cgrid, P.block, 0, s, pdl, P.ck));
  CK(launch(k_apply, dim3(1), dim3(1024), 0, s, pdl, P.ap));
  w->launches += 2;
  return DPF_OK;
}

template <class R>
static int launch_iteration(dpf_workspace* w, cudaStream_t s, bool with_check) {
  if (with_check) TRY(launch_check<R>(w, s, false));
  Plan<R> P = make_plan<R>(w);
  // event-bracketed (profiled) launches keep plain stream order
  const bool pdl = w->opts.pdl != 0 && !w->profile;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (w->profile) {
    TRY(ev_take(w, &e0));
    TRY(ev_take(w, &e1));
    TRY(ev_take(w, &e2));
    CK(cudaEventRecord(e0, s));
  }
  if constexpr (sizeof(R) == 4) {
    const bool ref = w->precision == DPF_FP32R;
    if (w->precision == DPF_MIXED) CK(launch(k_fwd_mixed, P.grid, P.block, P.smem, s, pdl, P.it));
    else if (w->direct)
      CK(launch(ref ? k_fwd<float, true, true> : k_fwd<float, false, true>, P.grid, P.block, 0, s, pdl, P.it));
    else if (w->pair_fwd) CK(launch(ref ? k_fwd2<true> : k_fwd2<false>, P.pgrid, P.block, P.smem, s, pdl, P.it));
    else CK(launch(ref ? k_fwd<float, true> : k_fwd<float, false>, P.grid, P.block, P.smem, s, pdl, P.it));
  } else {
    CK(launch(k_fwd<R>, P.grid, P.block, P.smem, s, pdl, P.it));
  }
  if (w->profile) CK(cudaEventRecord(e1, s));
  if constexpr (sizeof(R) == 4) {
    const bool ref = w->precision == DPF_FP32R;
    if (w->precision == DPF_MIXED) CK(launch(k_adj<float, true>, P.gridb, P.block, P.ysmem, s, pdl, P.itb));
    else if (w->direct)
      CK(launch(ref ? k_adj<float, false, true, true> : k_adj<float, false, false, true>, P.gridb, P.block, 0, s,
                pdl, P.itb));
    else if (w->pair_adj) CK(launch(ref ? k_adj2<true> : k_adj2<false>, P.pgridb, P.block, P.ysmem, s, pdl, P.itb));
    else CK(launch(ref ? k_adj<float, false, true> : k_adj<float, false, false>, P.gridb, P.block, P.ysmem, s, pdl,
                   P.itb));
  } else {
    CK(launch(k_adj<R>, P.gridb, P.block, P.ysmem, s, pdl, P.itb));
  }
  if (w->profile) {
    CK(cudaEventRecord(e2, s));
    const int i2 = (int)w->ev_used - 1;
    w->ev_fwd.push_back({i2 - 2, i2 - 1});
    w->ev_adj.push_back({i2 - 1, i2});
  }
  w->launches += 2;
  return DPF_OK;
}

static int launch_iteration_any(dpf_workspace* w, cudaStream_t s, bool with_check) {
  return w->precision == DPF_FP64 ? launch_iteration<double>(w, s, with_check)
                                  : launch_iteration<float>(w, s, with_check);
}
static int launch_check_any(dpf_workspace* w, cudaStream_t s, bool final_pass) {
  return w->precision == DPF_FP64 ? launch_check<double>(w, s, final_pass)
                                  : launch_check<float>(w, s, final_pass);
}

// Capture one check interval (FP64 test + check_every iterations) as a graph.
static int build_graph(dpf_workspace* w) {
  ws_drop_graph(w);
  cudaStream_t cs = w->cap_stream;
  const long long launches_before = w->launches;
  const bool prof = w->profile;
  w->profile = false;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = DPF_OK;
  for (int i = 0; i < w->opts.check_every && rc == DPF_OK; ++i) rc = launch_iteration_any(w, cs, i == 0);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (rc != DPF_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(DPF_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
  {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int kn = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      kn += (ty == cudaGraphNodeTypeKernel);
    }
    w->graph_kernels = kn;
  }
  w->launches = launches_before;
  w->profile = prof;
  e = cudaGraphInstantiate(&w->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    w->gexec = nullptr;
    return fail(DPF_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// State set-up shared by the solve and the evaluation entry points
// ---------------------------------------------------------------------------
struct StateIn {
  int K;
  bool host_io;
  bool enforce_fixed;  // solve: set-points override the given state; evaluation: state as given
  const double *va, *vm, *vmset, *p, *q;  // user layout [K][N] or NULL
  const double *va0, *vm0;                 // one start [N] shared by every case, or NULL
  const int32_t* outage;
};

static void choose_shape(dpf_workspace* w, const dpf_solve_opts* o, int K) {
  int lanes = (o && o->lanes > 0) ? o->lanes : std::min(32, pow2ceil(K));
  if (lanes > 32) lanes = 32;
  lanes = pow2ceil(lanes);
  w->lanes = lanes;
  // FP32 solve loop over >= 64 cases at 32 lanes: two cases per thread
  w->pairs = o && (o->precision == DPF_FP32 || o->precision == DPF_FP32R) && lanes == 32 && K >= 64 &&
             o->pair_cases != 0;
  w->pair_fwd = w->pairs && (o->pair_cases & 1);
  w->pair_adj = w->pairs && (o->pair_cases & 2);
  const int tile = w->pairs ? 64 : lanes;
  w->Kp = (K + tile - 1) / tile * tile;
  w->warps = (o && o->warps > 0) ? std::min(o->warps, 8) : 8;
  const int rpw = 32 / lanes;
  w->gx = w->Kp / lanes;
  const int rows_per_cta = w->warps * rpw;
  const int gy_max = std::max(1, (w->y->n + rows_per_cta - 1) / rows_per_cta);
  int gy;
  if (o && o->row_blocks > 0) gy = o->row_blocks;
  else gy = (num_sms() * 8 + w->gx - 1) / w->gx;
  gy = std::max(1, std::min(std::min(gy, gy_max), 65535));
  const int n = w->y->n;
  const std::vector<int32_t>& rp = w->y->irow_ptr;
  const std::vector<int32_t>& prp = w->y->iprow_ptr;  // padded rows: the staged entries
  const std::vector<int32_t>& col = w->y->icol;
  const int prec = o ? o->precision : w->precision;
  // a single-case FP32 solve reads its Y rows from global memory (no reuse to stage for)
  w->direct = o && lanes == 1 && (prec == DPF_FP32 || prec == DPF_FP32R) && o->plain == 0 && o->stage_y == 0;
  const bool fp64 = prec == DPF_FP64;        // FP64 adjoint (and forward)
  const bool mixed = prec == DPF_MIXED;      // FP64 forward, FP32 adjoint
  const bool refined = prec == DPF_FP32R;    // FP32 iterations on FP64 references
  const bool fp64_fwd = fp64 || mixed;       // the forward pass stages FP64 Y rows
  // bytes of one staged window row: the case tile's line of V (not in mixed mode)
  const bool stage_v = o && o->stage_v && !mixed;
  const int line = !stage_v ? 0 : w->pair_fwd ? 512 : (lanes == 32 ? 32 * (fp64 ? 16 : 8) : 0);
  if (w->direct) {  // no staged rows: any row-block size fits
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_adj<float, false, false, true>,
                                                  w->warps * 32, 0);
    cudaGetLastError();
    if (!(o && o->row_blocks > 0)) gy = std::min(gy_max, num_sms() * std::max(1, occ));
    const int rpb = (n + gy - 1) / gy;
    w->rpb = w->rpb_b = rpb;
    w->gy = w->gy_b = (n + rpb - 1) / rpb;
    w->ysmem = w->ysmem_b = w->smem = 0;
    w->staged = false;
    w->h_wlo.assign(w->gy, 0);
    w->h_whi.assign(w->gy, 0);
    return;
  }
  // shrink row blocks until the staged Y rows (and the V window) fit
  for (int tries = 0;; ++tries) {
    const int rpb = (n + gy - 1) / gy;
    int mx = 0, wmax = 0;
    for (int r0 = 0; r0 < n; r0 += rpb) {
      const int r1 = std::min(n, r0 + rpb);
      mx = std::max(mx, prp[r1] - prp[r0]);
      int lo = r0, hi = r1 - 1;
      for (int q = rp[r0]; q < rp[r1]; ++q) { lo = std::min(lo, col[q]); hi = std::max(hi, col[q]); }
      wmax = std::max(wmax, hi - lo + 1);
    }
    const int ybytes = ysmem_bytes(rpb, mx, fp64_fwd);
    const int wbytes = line * wmax;
    const bool fits = ybytes + wbytes <= 150 * 1024;
    // (staged Y rows above ~32 KB would cap the resident CTAs per SM)
    if ((fits && line > 0) || (line == 0 && ybytes <= 32 * 1024) || gy >= 65535 || rpb <= 1 || tries >= 6) {
      w->gy = (n + rpb - 1) / rpb;
      w->rpb = rpb;
      w->ysmem = ybytes;
      w->staged = line > 0 && fits;
      w->smem = ybytes + (w->staged ? wbytes : 0);
      break;
    }
    gy = std::min(65535, gy * 2);
  }
  // Row blocks per pass, sized so that each grid is a whole number of waves
  // of resident CTAs (a partial last wave leaves SMs idle at the tail).
  auto seg_nnz = [&](int rpb_) {
    int mx = 0;
    for (int r0 = 0; r0 < n; r0 += rpb_) mx = std::max(mx, prp[std::min(n, r0 + rpb_)] - prp[r0]);
    return mx;
  };
  auto aligned = [&](int gx_k, int slots, int gy0) {
    if (slots <= 0) return gy0;
    const int waves = std::max(1, (int)((double)gx_k * gy0 / slots + 0.5));
    int g_ = std::max(1, std::min(n, (int)((long long)waves * slots / gx_k)));
    const int rpb_ = (n + g_ - 1) / g_;
    return (n + rpb_ - 1) / rpb_;
  };
  const bool auto_rb = !(o && o->row_blocks > 0);
  const int block = w->warps * 32;
  const int sms = num_sms();
  w->gy_b = w->gy;
  if (auto_rb && !w->staged) {
    int occ_f = 0, occ_b = 0;
    const void* kf = fp64          ? (const void*)k_fwd<double>
                     : mixed       ? (const void*)k_fwd_mixed
                     : w->pair_fwd ? (refined ? (const void*)k_fwd2<true> : (const void*)k_fwd2<false>)
                     : refined     ? (const void*)k_fwd<float, true>
                                   : (const void*)k_fwd<float>;
    const void* kb = fp64          ? (const void*)k_adj<double>
                     : mixed       ? (const void*)k_adj<float, true>
                     : w->pair_adj ? (refined ? (const void*)k_adj2<true> : (const void*)k_adj2<false>)
                     : refined     ? (const void*)k_adj<float, false, true>
                                   : (const void*)k_adj<float>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, kf, block, w->smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, kb, block, w->smem);
    cudaGetLastError();  // a failed query only disables the alignment
    const int gxf = w->pair_fwd ? w->Kp / 64 : w->gx;
    const int gxb = w->pair_adj ? w->Kp / 64 : w->gx;
    const int gyf = aligned(gxf, occ_f * sms, w->gy);
    w->gy_b = aligned(gxb, occ_b * sms, w->gy);
    if (gyf != w->gy) {
      w->rpb = (n + gyf - 1) / gyf;
      w->gy = (n + w->rpb - 1) / w->rpb;
      w->ysmem = ysmem_bytes(w->rpb, seg_nnz(w->rpb), fp64_fwd);
      w->smem = w->ysmem;
    }
  }
  w->rpb_b = (n + w->gy_b - 1) / w->gy_b;
  w->gy_b = (n + w->rpb_b - 1) / w->rpb_b;
  w->ysmem_b = ysmem_bytes(w->rpb_b, seg_nnz(w->rpb_b), fp64);  // the adjoint's own precision
  w->h_wlo.assign(w->gy, 0);
  w->h_whi.assign(w->gy, 0);
  for (int b = 0; b < w->gy; ++b) {
    const int r0 = b * w->rpb, r1 = std::min(n, r0 + w->rpb);
    int lo = r0, hi = r1 - 1;
    for (int q = rp[r0]; q < rp[r1]; ++q) { lo = std::min(lo, col[q]); hi = std::max(hi, col[q]); }
    w->h_wlo[b] = lo;
    w->h_whi[b] = hi;
  }
}

// Device copies of the row-block windows (after choose_shape), and zeroed
// per-tile counters for the forward pass's scheduler.
static int upload_windows(dpf_workspace* w, cudaStream_t s) {
  const int tiles = std::max(w->Kp / std::max(1, w->lanes), w->Kp / 64 + 1);
  const int groups = (w->gy + SCHED_GROUP - 1) / SCHED_GROUP;
  const int cnts = tiles * (1 + groups);  // tile counters, then per (tile, group) counters
  if (cnts > w->cap_tiles) {
    dfree(w->tile_cnt);
    w->cap_tiles = 0;
    TRY(dalloc(&w->tile_cnt, cnts));
    w->cap_tiles = cnts;
  }
  w->tiles = tiles;
  CK(cudaMemsetAsync(w->tile_cnt, 0, (size_t)w->cap_tiles * sizeof(unsigned int), s));
  const size_t part = (size_t)(w->gy + groups) * w->Kp;  // row-block partials, then group sums
  if (part > w->cap_part) {
    dfree(w->loss_part);
    w->cap_part = 0;
    TRY(dalloc((char**)&w->loss_part, part * 8));
    w->cap_part = part;
  }
  if (w->gy > w->cap_wblocks) {
    dfree(w->d_wlo);
    dfree(w->d_whi);
    w->cap_wblocks = 0;
    TRY(dalloc(&w->d_wlo, w->gy));
    TRY(dalloc(&w->d_whi, w->gy));
    w->cap_wblocks = w->gy;
  }
  CK(cudaMemcpyAsync(w->d_wlo, w->h_wlo.data(), w->gy * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->d_whi, w->h_whi.data(), w->gy * 4, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // host vectors may change at the next choose_shape
  return DPF_OK;
}

template <class R>
static int set_smem_attr(int bytes) {
  if (bytes > 48 * 1024) {
    CK(cudaFuncSetAttribute(k_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    CK(cudaFuncSetAttribute(k_adj<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if constexpr (sizeof(R) == 4) {
      CK(cudaFuncSetAttribute(k_fwd2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_adj2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_fwd2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_adj2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_fwd<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_adj<float, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_fwd_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      CK(cudaFuncSetAttribute(k_adj<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    }
  }
  return DPF_OK;
}

// Copy an input (user layout) into the internal layout buffer `dst`.
static int to_internal(dpf_workspace* w, const double* src, bool host_io, double* stage, double* dst,
                       cudaStream_t s) {
  const dpf_ybus* y = w->y;
  const double* dsrc = src;
  if (host_io) {
    CK(cudaMemcpyAsync(stage, src, (size_t)w->K * y->n * 8, cudaMemcpyHostToDevice, s));
    dsrc = stage;
  }
  dim3 g((y->n + 31) / 32, (w->K + 31) / 32), b(32, 8);
  k_to_internal<<<g, b, 0, s>>>(dsrc, dst, w->K, y->n, w->Kp, y->dev.iperm);
  CKLAUNCH();
  w->launches++;
  return DPF_OK;
}

static int to_user(dpf_workspace* w, const double* src, bool host_io, double* stage, double* dst,
                   cudaStream_t s) {
  const dpf_ybus* y = w->y;
  double* ddst = host_io ? stage : dst;
  dim3 g((y->n + 31) / 32, (w->K + 31) / 32), b(32, 8);
  k_to_user<<<g, b, 0, s>>>(src, ddst, w->K, y->n, w->Kp, y->dev.iperm);
  CKLAUNCH();
  w->launches++;
  if (host_io) CK(cudaMemcpyAsync(dst, stage, (size_t)w->K * y->n * 8, cudaMemcpyDeviceToHost, s));
  return DPF_OK;
}

// Validate an outage list against the grid (copies it to the host).
static int check_outages(dpf_workspace* w, const int32_t* outage, bool host_io, cudaStream_t s) {
  const dpf_ybus* y = w->y;
  std::vector<int32_t> h(w->K);
  if (host_io) {
    memcpy(h.data(), outage, (size_t)w->K * 4);
  } else {
    CK(cudaMemcpyAsync(h.data(), outage, (size_t)w->K * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  for (int k = 0; k < w->K; ++k) {
    const int l = h[k];
    if (l < -1 || l >= y->m) return fail(DPF_E_INVALID, "case %d: outage index %d out of range", k, l);
    if (l >= 0 && y->bridge[l]) return fail(DPF_E_ISLANDED, "case %d: removing branch %d islands the grid", k, l);
  }
  return DPF_OK;
}

template <class R>
static int init_state(dpf_workspace* w, const StateIn& in, cudaStream_t s) {
  const dpf_ybus* y = w->y;
  const DeviceYbus& d = y->dev;
  const bool hio = in.host_io;
  // inputs to the internal layout
  double* va_t = nullptr;
  double* vm_t = nullptr;
  double* vms_t = nullptr;
  bool shared = false;
  if (in.va0 && in.vm0) {  // one state for every case: [N] in internal bus order
    const double* src[2] = {in.va0, in.vm0};
    double* stage[2] = {w->st_a, w->st_b};
    double* dst[2] = {w->tmp_a, w->tmp_b};
    for (int j = 0; j < 2; ++j) {
      const double* d = src[j];
      if (hio) {
        CK(cudaMemcpyAsync(stage[j], src[j], (size_t)y->n * 8, cudaMemcpyHostToDevice, s));
        d = stage[j];
      }
      k_to_internal<<<dim3((y->n + 31) / 32, 1), dim3(32, 8), 0, s>>>(d, dst[j], 1, y->n, 1, y->dev.iperm);
      CKLAUNCH();
      w->launches++;
    }
    va_t = w->tmp_a;
    vm_t = w->tmp_b;
    shared = true;
  } else if (in.va && in.vm) {
    TRY(to_internal(w, in.va, hio, w->st_a, w->tmp_a, s));
    TRY(to_internal(w, in.vm, hio, w->st_b, w->tmp_b, s));
    va_t = w->tmp_a;
    vm_t = w->tmp_b;
  }
  if (in.vmset) {
    TRY(to_internal(w, in.vmset, hio, w->st_c, w->tmp_c, s));
    vms_t = w->tmp_c;
  }
  if ((in.p == nullptr) != (in.q == nullptr))
    return fail(DPF_E_INVALID, "p_spec and q_spec must be given together");
  w->spec_per_case = (in.p != nullptr);
  if (w->spec_per_case) {
    TRY(to_internal(w, in.p, hio, w->st_a, w->p64, s));
    TRY(to_internal(w, in.q, hio, w->st_b, w->q64, s));
  }
  InitArgs<R> ia;
  memset(&ia, 0, sizeof ia);
  ia.N = y->n;
  ia.K = w->K;
  ia.Kp = w->Kp;
  ia.enforce_fixed = in.enforce_fixed ? 1 : 0;
  ia.type = d.type;
  ia.vmset_grid = d.vmset;
  ia.vms_t = vms_t;
  ia.va_t = va_t;
  ia.vm_t = vm_t;
  ia.shared_start = shared ? 1 : 0;
  ia.va_slack = y->va_slack;
  ia.p64 = w->spec_per_case ? w->p64 : nullptr;
  ia.q64 = w->spec_per_case ? w->q64 : nullptr;
  ia.p = (R*)w->p;
  ia.q = (R*)w->q;
  ia.ms = (typename Prec<R>::MS*)w->ms;
  ia.V = (typename Prec<R>::C*)w->V;
  ia.os = (Mom<R>*)w->os;
  const size_t E = (size_t)y->n * w->Kp;
  const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
  k_init<R><<<std::max(nb, 1), 256, 0, s>>>(ia);
  CKLAUNCH();
  w->launches++;
  if constexpr (sizeof(R) == 4) {
    if (w->precision == DPF_MIXED) {  // FP64 voltages for the mixed forward pass
      k_mixed_v64<<<std::max(nb, 1), 256, 0, s>>>((const float4*)w->ms, (double2*)w->V, E);
      CKLAUNCH();
      w->launches++;
    }
  }

  // per-case state and N-1 corrections
  w->has_outage = (in.outage != nullptr);
  const int32_t* outage_dev = nullptr;
  if (in.outage) {
    TRY(check_outages(w, in.outage, hio, s));
    if (hio) {
      CK(cudaMemcpyAsync(w->outage_dev, in.outage, (size_t)w->K * 4, cudaMemcpyHostToDevice, s));
      outage_dev = w->outage_dev;
    } else {
      outage_dev = in.outage;
    }
  }
  CaseInitArgs<R> ca;
  memset(&ca, 0, sizeof ca);
  ca.K = w->K;
  ca.Kp = w->Kp;
  ca.outage = outage_dev;
  ca.br_f = d.br_f;
  ca.br_t = d.br_t;
  ca.br_r = d.br_r;
  ca.br_x = d.br_x;
  ca.br_bch = d.br_bch;
  ca.br_tap = d.br_tap;
  ca.of = w->of;
  ca.ot = w->ot;
  ca.yff = (typename Prec<R>::C*)w->yff;
  ca.yft = (typename Prec<R>::C*)w->yft;
  ca.ytt = (typename Prec<R>::C*)w->ytt;
  ca.yff64 = w->yff64;
  ca.yft64 = w->yft64;
  ca.ytt64 = w->ytt64;
  ca.active = w->active;
  ca.iters = w->iters;
  ca.status = w->status;
  ca.lr = w->lr;
  ca.best = w->best;
  ca.bad = w->bad;
  ca.cool = w->cool;
  ca.step_size = (R*)w->step_size;
  ca.isbc2 = (R*)w->isbc2;
  ca.b1t = w->b1t;
  ca.b2t = w->b2t;
  ca.cand = w->cand;
  ca.mx32 = w->mx32;
  ca.maxmis = w->maxmis;
  ca.loss64 = w->loss64;
  ca.lr0 = w->opts.lr;
  ca.beta1 = w->opts.beta1;
  ca.beta2 = w->opts.beta2;
  ca.opt = w->opts.optimizer;
  k_case_init<R><<<(w->Kp + 255) / 256, 256, 0, s>>>(ca);
  CKLAUNCH();
  w->launches++;
  CK(cudaMemcpyAsync(w->n_active, &w->K, 4, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // &w->K is host memory that may change later
  return DPF_OK;
}

static int validate_opts(const dpf_solve_opts* o) {
  if (!(o->lr > 0) || !(o->beta1 >= 0 && o->beta1 < 1) || !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps >= 0))
    return fail(DPF_E_INVALID, "invalid Adam parameters");
  if (o->sched < DPF_SCHED_CONST || o->sched > DPF_SCHED_STEP) return fail(DPF_E_INVALID, "unknown scheduler");
  if (o->optimizer < DPF_OPT_ADAM || o->optimizer > DPF_OPT_RMSPROP) return fail(DPF_E_INVALID, "unknown optimizer");
  if (!(o->momentum >= 0 && o->momentum < 1) || !(o->alpha >= 0 && o->alpha < 1))
    return fail(DPF_E_INVALID, "momentum and alpha must be in [0, 1)");
  if (o->sched == DPF_SCHED_PLATEAU && (!(o->factor > 0 && o->factor < 1) || o->patience < 0 || o->cooldown < 0))
    return fail(DPF_E_INVALID, "invalid plateau parameters");
  if (o->sched == DPF_SCHED_STEP && (o->step_size < 1 || !(o->gamma > 0)))
    return fail(DPF_E_INVALID, "invalid StepLR parameters");
  if (o->max_iter < 0 || o->check_every < 1 || !(o->tol >= 0))
    return fail(DPF_E_INVALID, "invalid max_iter / check_every / tol");
  if (o->precision != DPF_FP32 && o->precision != DPF_FP64 && o->precision != DPF_MIXED &&
      o->precision != DPF_FP32R)
    return fail(DPF_E_INVALID, "unknown precision");
  if (!(o->gate >= 0.0)) return fail(DPF_E_INVALID, "gate must be >= 0");
  if (o->pdl != 0 && o->pdl != 1) return fail(DPF_E_INVALID, "pdl must be 0 or 1");
  if (o->dc_start != 0 && o->dc_start != 1) return fail(DPF_E_INVALID, "dc_start must be 0 or 1");
  if (o->dc_start && (!(o->dc_tol > 0 && o->dc_tol < 1e300) || o->dc_max_iter < 1))
    return fail(DPF_E_INVALID, "dc_start needs dc_tol > 0 and dc_max_iter >= 1");
  if (o->stage_y != 0 && o->stage_y != 1) return fail(DPF_E_INVALID, "stage_y must be 0 or 1");
  if (o->refresh_every < 0) return fail(DPF_E_INVALID, "refresh_every must be >= 0");
  if (o->lanes < 0 || o->lanes > 32 || o->warps < 0 || o->warps > 8 || o->row_blocks < 0)
    return fail(DPF_E_INVALID, "invalid launch shape (lanes 0..32, warps 0..8, row_blocks >= 0)");
  return DPF_OK;
}

static int common_checks(const dpf_ybus* y, dpf_workspace* w, int K) {
  if (!y || !w) return fail(DPF_E_INVALID, "NULL handle");
  if (w->y != y) return fail(DPF_E_INVALID, "workspace was created for another Y_bus");
  if (!y->dev.ready) return fail(DPF_E_STATE, "Y_bus is not on the device");
  if (K < 1) return fail(DPF_E_INVALID, "n_case must be >= 1");
  // the staged SpMV addresses a gathered element by a 32-bit offset bus * Kp
  if ((uint64_t)y->n * (uint64_t)(K + 64) >= (1ull << 32))
    return fail(DPF_E_UNSUPPORTED, "n_bus * n_case must stay below 2^32 (split the batch)");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != y->dev.device) return fail(DPF_E_STATE, "current device %d differs from the Y_bus device %d", dev, y->dev.device);
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// DC approximation (batched Jacobi-preconditioned CG, FP64); the solution x
// is left in w->tmp_a ([N][Kp]); needs the specification and outages staged by
// init_state.
// ---------------------------------------------------------------------------
__global__ void k_dc_set_count(int32_t* n, int K) { *n = K; }

// B' x = P for every case (shift = false), or the outage shift of the cases'
// start angles in the master state (shift = true; x0 = 0, right-hand side
// from k_dc_flow).  x ends in tmp_a as FP64.  T = float2: double-float
// vectors (8 bytes per element, in the FP64 buffers); T = float: FP32 vectors,
// all but z in V64's 16 bytes per element.
template <class T>
static int dc_run_t(dpf_workspace* w, const int32_t* outage_dev, double tol, int max_iter, cudaStream_t s,
                    bool shift) {
  const dpf_ybus* y = w->y;
  const DeviceYbus& d = y->dev;
  const int Kp = w->Kp;
  DCArgs<T> a;
  memset(&a, 0, sizeof a);
  a.N = y->n;
  a.Kp = Kp;
  a.lanes = w->lanes;
  a.K = w->K;
  a.rp = d.row_ptr;
  a.col = d.col;
  a.bval = d.dcval;
  a.dpos = d.dpos;
  a.dinv = d.dcinv;
  a.type = d.type;
  a.spec_per_case = w->spec_per_case ? 1 : 0;
  a.pspec = w->spec_per_case ? w->p64 : d.p64;
  a.va_slack = y->va_slack;
  a.of = w->has_outage ? w->of : nullptr;
  a.ot = w->has_outage ? w->ot : nullptr;
  const size_t E = (size_t)y->n * Kp;
  if constexpr (sizeof(T) == 8) {
    a.x = (T*)w->tmp_a;
    a.r = (T*)w->tmp_b;
    a.z = (T*)w->tmp_c;
    a.p = (T*)w->V64;  // the two direction buffers share V64's 16 B/element
    a.p_new = (T*)w->V64 + E;
    a.q = (T*)w->sbuf;
  } else {
    a.p = (T*)w->V64;
    a.p_new = (T*)w->V64 + E;
    a.x = (T*)w->V64 + 2 * E;
    a.r = (T*)w->V64 + 3 * E;
    a.z = (T*)w->tmp_c;
    a.q = (T*)w->sbuf;
  }
  a.rpb = w->rpb;
  a.tile_cnt = w->tile_cnt;
  double* c = w->dcs;
  a.rz = c;
  a.rzn = c + Kp;
  a.pq = c + 2 * (size_t)Kp;
  a.rr = c + 3 * (size_t)Kp;
  a.rr0 = c + 4 * (size_t)Kp;
  a.beta = c + 5 * (size_t)Kp;
  a.res = c + 6 * (size_t)Kp;
  a.ob = c + 7 * (size_t)Kp;
  a.flow = shift ? c + 8 * (size_t)Kp : nullptr;
  if (shift) a.va_slack = 0.0;  // x is an angle change: 0 at the slack buses
  a.active = w->dci;
  a.iters = w->dci + Kp;
  a.n_active = w->dci + 2 * (size_t)Kp;
  a.tol2 = tol * tol;
  const dim3 grid(Kp / w->lanes, w->gy), block(w->warps * 32);
  const int cb = (Kp + 255) / 256;
  const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
  k_dc_case_init<T><<<cb, 256, 0, s>>>(a, outage_dev, d.br_x, d.br_tap);
  if (shift) {
    if (!a.of) return fail(DPF_E_INVALID, "the outage shift needs outages");
    if (w->precision == DPF_FP64)
      k_dc_flow<double><<<cb, 256, 0, s>>>((const double2*)w->ms, a.of, a.ot, a.ob, c + 8 * (size_t)Kp, w->K, Kp);
    else
      k_dc_flow<float><<<cb, 256, 0, s>>>((const float4*)w->ms, a.of, a.ot, a.ob, c + 8 * (size_t)Kp, w->K, Kp);
  }
  k_dc_set_count<<<1, 1, 0, s>>>(a.n_active, w->K);
  k_dc_x0<T><<<std::max(nb, 1), 256, 0, s>>>(a);
  k_dc_start<T><<<grid, block, 0, s>>>(a);
  CKLAUNCH();
  w->launches += shift ? 5 : 4;
  for (int it = 0; it < max_iter; ++it) {
    k_dc_spmv_dir<T><<<grid, block, 0, s>>>(a);
    k_dc_update_case<T><<<grid, block, 0, s>>>(a);
    CKLAUNCH();
    w->launches += 2;
    std::swap(a.p, a.p_new);
    if ((it & 15) == 15 || it == max_iter - 1) {
      CK(cudaMemcpyAsync(w->h_dc_nact, a.n_active, 4, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*w->h_dc_nact == 0) break;
    }
  }
  k_dc_widen<T><<<std::max(nb, 1), 256, 0, s>>>(a.x, w->tmp_a, E);  // the FP64 solution
  CKLAUNCH();
  w->launches++;
  return DPF_OK;
}

// Relative residuals of 1e-5 and above run on FP32 vectors.
static int dc_run(dpf_workspace* w, const int32_t* outage_dev, double tol, int max_iter, cudaStream_t s,
                  bool shift = false) {
  return tol >= 1e-5 ? dc_run_t<float>(w, outage_dev, tol, max_iter, s, shift)
                     : dc_run_t<float2>(w, outage_dev, tol, max_iter, s, shift);
}

extern "C" int dpf_dc_solve(const dpf_ybus* y, dpf_workspace* w, int32_t n_case, const double* p_spec,
                            const int32_t* outage, double tol, int32_t max_iter, double* va, int32_t* iters,
                            double* rel_residual, void* stream) {
  dpf::Range nvtx_range("dpf_dc_solve");
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  TRY(common_checks(y, w, n_case));
  if (!va) return fail(DPF_E_INVALID, "dpf_dc_solve: va is required");
  if (!(tol > 0) || max_iter < 1) return fail(DPF_E_INVALID, "dpf_dc_solve: tol > 0 and max_iter >= 1 required");
  w->begun = false;
  w->pid_ready = false;
  ws_drop_graph(w);
  dpf_default_opts(&w->opts);
  w->opts.precision = DPF_FP64;
  w->precision = DPF_FP64;
  w->K = n_case;
  choose_shape(w, nullptr, n_case);
  TRY(upload_windows(w, s));
  TRY(ws_reserve(w, w->Kp, 0));
  StateIn in;
  memset(&in, 0, sizeof in);
  in.K = n_case;
  in.enforce_fixed = true;
  in.p = p_spec;
  in.q = p_spec;  // (the DC model reads only P)
  in.outage = outage;
  TRY(init_state<double>(w, in, s));
  TRY(dc_run(w, outage, tol, max_iter, s));
  TRY(to_user(w, w->tmp_a, false, nullptr, va, s));
  if (iters) CK(cudaMemcpyAsync(iters, w->dci + w->Kp, (size_t)n_case * 4, cudaMemcpyDeviceToDevice, s));
  if (rel_residual)
    CK(cudaMemcpyAsync(rel_residual, w->dcs + 6 * (size_t)w->Kp, (size_t)n_case * 8, cudaMemcpyDeviceToDevice, s));
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// Solve
// ---------------------------------------------------------------------------
extern "C" int dpf_solve_begin(const dpf_ybus* y, dpf_workspace* w, const dpf_batch* b,
                               const dpf_solve_opts* o, void* stream) {
  dpf::Range nvtx_range("dpf_solve_begin");
  clear_error();
  if (!b || !o) return fail(DPF_E_INVALID, "dpf_solve_begin: NULL argument");
  TRY(common_checks(y, w, b->n_case));
  TRY(validate_opts(o));
  if ((b->va_start == nullptr) != (b->vm_start == nullptr))
    return fail(DPF_E_INVALID, "va_start and vm_start must be given together");
  if (!o->flat_start && !b->va_start && (!b->va || !b->vm)) return fail(DPF_E_INVALID, "warm start needs va and vm");
  cudaStream_t s = (cudaStream_t)stream;
  w->begun = false;
  w->pid_ready = false;
  ws_drop_graph(w);
  w->opts = *o;
  w->K = b->n_case;
  w->precision = o->precision;
  w->use_local_y = false;
  choose_shape(w, o, w->K);
  TRY(upload_windows(w, s));
  TRY(w->precision == DPF_FP64 ? set_smem_attr<double>(std::max(w->smem, w->ysmem_b))
                               : set_smem_attr<float>(std::max(w->smem, w->ysmem_b)));
  TRY(ws_reserve(w, w->Kp, b->host_io ? (size_t)w->K * y->n : 0));
  StateIn in;
  memset(&in, 0, sizeof in);
  in.K = w->K;
  in.host_io = b->host_io != 0;
  in.enforce_fixed = true;
  if (!o->flat_start) {
    in.va = b->va;
    in.vm = b->vm;
    in.va0 = b->va_start;
    in.vm0 = b->vm_start;
  }
  in.vmset = b->vm_set;
  in.p = b->p_spec;
  in.q = b->q_spec;
  in.outage = b->outage;
  TRY(w->precision == DPF_FP64 ? init_state<double>(w, in, s) : init_state<float>(w, in, s));
  // angles from the DC approximation (flat start) or shifted by the DC angle
  // change of each case's outage (warm start); |V| as initialised
  const bool dc_shift = o->dc_start && !o->flat_start && b->outage;
  if ((o->flat_start && o->dc_start) || dc_shift) {
    const int32_t* od = b->outage ? (b->host_io ? w->outage_dev : b->outage) : nullptr;
    TRY(dc_run(w, od, o->dc_tol, o->dc_max_iter, s, dc_shift));
    const size_t E = (size_t)y->n * w->Kp;
    const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
    const int add = dc_shift ? 1 : 0;
    if (w->precision == DPF_FP64)
      k_dc_apply<double><<<nb, 256, 0, s>>>(w->tmp_a, (double2*)w->ms, (double2*)w->V, y->dev.type, y->n, w->K, w->Kp,
                                            add);
    else
      k_dc_apply<float><<<nb, 256, 0, s>>>(w->tmp_a, (float4*)w->ms, (float2*)w->V, y->dev.type, y->n, w->K, w->Kp,
                                           add);
    if (w->precision == DPF_MIXED) k_mixed_v64<<<nb, 256, 0, s>>>((const float4*)w->ms, (double2*)w->V, E);
    CKLAUNCH();
    w->launches += (w->precision == DPF_MIXED) ? 2 : 1;
  }
  if (w->direct) {  // padded entries of the direct view
    const size_t np = (size_t)y->iprow_ptr[y->n];
    if (np > w->cap_pent) {
      dfree(w->pent);
      w->cap_pent = 0;
      TRY(dalloc(&w->pent, np));
      w->cap_pent = np;
    }
    const int nb = (int)std::min<size_t>((np + 255) / 256, (size_t)num_sms() * 16);
    k_pad_entries<<<std::max(nb, 1), 256, 0, s>>>(y->dev.ppos, y->dev.ent32, (int)np, w->pent);
    CKLAUNCH();
    w->launches++;
  }
  if (w->precision == DPF_FP32R) {  // (after the DC start, which uses these buffers)
    const size_t E = (size_t)y->n * w->Kp;
    const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
    k_ref_init<<<std::max(nb, 1), 256, 0, s>>>(y->dev.type, w->spec_per_case ? (const float*)w->p : y->dev.p32,
                                                w->spec_per_case ? (const float*)w->q : y->dev.q32,
                                                w->spec_per_case ? 1 : 0, w->Kp, E, (float2*)w->cbuf,
                                                (float4*)w->sbuf);
    CKLAUNCH();
    w->launches++;
  }
  w->t_done = 0;
  w->begun = true;
  return DPF_OK;
}

extern "C" int dpf_solve_iterate(dpf_workspace* w, int32_t n_iter, void* stream) {
  dpf::Range nvtx_range("dpf_solve_iterate");
  clear_error();
  if (!w || !w->begun) return fail(DPF_E_STATE, "dpf_solve_iterate before dpf_solve_begin");
  if (n_iter < 0) return fail(DPF_E_INVALID, "n_iter must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  n_iter = std::min(n_iter, w->opts.max_iter - w->t_done);
  const int ce = w->opts.check_every;
  while (n_iter > 0) {
    if (w->opts.use_graph && !w->profile && w->t_done % ce == 0 && n_iter >= ce) {
      if (!w->gexec) TRY(build_graph(w));
      CK(cudaGraphLaunch(w->gexec, s));
      w->launches += w->graph_kernels;
      w->t_done += ce;
      n_iter -= ce;
    } else {
      TRY(launch_iteration_any(w, s, w->t_done % ce == 0));
      w->t_done += 1;
      n_iter -= 1;
    }
  }
  return DPF_OK;
}

extern "C" int dpf_active_count(dpf_workspace* w, int32_t* n_active, void* stream) {
  if (!w || !n_active) return fail(DPF_E_INVALID, "dpf_active_count: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(w->h_n_active, w->n_active, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *n_active = *w->h_n_active;
  return DPF_OK;
}

extern "C" int dpf_profile_enable(dpf_workspace* w, int32_t on) {
  if (!w) return fail(DPF_E_INVALID, "dpf_profile_enable: NULL workspace");
  w->profile = on != 0;
  w->ev_used = 0;
  w->ev_fwd.clear();
  w->ev_adj.clear();
  return DPF_OK;
}

extern "C" int dpf_kernel_times(dpf_workspace* w, double* fwd_ms, double* adj_ms, int32_t* n_fwd, int32_t* n_adj,
                                void* stream) {
  if (!w) return fail(DPF_E_INVALID, "dpf_kernel_times: NULL workspace");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  double tf = 0.0, ta = 0.0;
  for (auto& pr : w->ev_fwd) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, w->ev_pool[pr.first], w->ev_pool[pr.second]));
    tf += ms;
  }
  for (auto& pr : w->ev_adj) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, w->ev_pool[pr.first], w->ev_pool[pr.second]));
    ta += ms;
  }
  if (fwd_ms) *fwd_ms = tf;
  if (adj_ms) *adj_ms = ta;
  if (n_fwd) *n_fwd = (int32_t)w->ev_fwd.size();
  if (n_adj) *n_adj = (int32_t)w->ev_adj.size();
  return DPF_OK;
}

extern "C" int dpf_kernel_launches(const dpf_workspace* w, int64_t* n) {
  if (!w || !n) return fail(DPF_E_INVALID, "dpf_kernel_launches: NULL argument");
  *n = w->launches;
  return DPF_OK;
}

// Read-bandwidth probe: every thread sums its 16-byte words (four loads in
// flight per step); the sums feed a store no input can trigger, so the loads
// cannot be dropped.
__global__ void __launch_bounds__(256) k_read_probe(const float4* __restrict__ p, size_t n4, int passes,
                                                    float* __restrict__ sink) {
  float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int pass = 0; pass < passes; ++pass) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    const float4 v0 = __ldcg(p + i), v1 = __ldcg(p + i + stride), v2 = __ldcg(p + i + 2 * stride),
                 v3 = __ldcg(p + i + 3 * stride);
    ax += (v0.x + v1.x) + (v2.x + v3.x);
    ay += (v0.y + v1.y) + (v2.y + v3.y);
    az += (v0.z + v1.z) + (v2.z + v3.z);
    aw += (v0.w + v1.w) + (v2.w + v3.w);
  }
  for (; i < n4; i += stride) {
    const float4 v = __ldcg(p + i);
    ax += v.x; ay += v.y; az += v.z; aw += v.w;
  }
  }
  const float t = (ax + ay) + (az + aw);
  if (t == -1.2345e-38f) sink[blockIdx.x] = t;  // never true for the probe's data
}

extern "C" int dpf_read_bandwidth(const void* buf, int64_t bytes, int32_t reps, double* gbs, void* stream) {
  clear_error();
  if (!buf || !gbs || bytes <= 0 || reps < 1) return fail(DPF_E_INVALID, "dpf_read_bandwidth: bad argument");
  if (((uintptr_t)buf & 15) != 0 || (bytes & 15) != 0)
    return fail(DPF_E_INVALID, "dpf_read_bandwidth: buffer and size must be multiples of 16 bytes");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n4 = (size_t)bytes / 16;
  const int grid = num_sms() * 8;
  // buffers that fit the L2 are read several times per launch (>= 256 MB per
  // launch), so that launch gaps do not dilute the measurement
  const int passes = (int)std::max<int64_t>(1, std::min<int64_t>(64, (256ll << 20) / bytes));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = DPF_OK;
  for (int r = 0; r < 2; ++r) k_read_probe<<<grid, 256, 0, s>>>((const float4*)buf, n4, passes, nullptr);
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) k_read_probe<<<grid, 256, 0, s>>>((const float4*)buf, n4, passes, nullptr);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) rc = fail(DPF_E_CUDA, "dpf_read_bandwidth: %s", cudaGetErrorString(e));
  else *gbs = (double)bytes * passes * reps / (ms * 1e-3) / 1e9;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// Grid-wide barrier probe: `reps` barriers of a cooperative grid (all CTAs
// co-resident, guaranteed by the cooperative launch, which fails rather than
// waits if they cannot be).
__global__ void __launch_bounds__(256) k_barrier_probe(int reps, int* __restrict__ sink) {
  cooperative_groups::grid_group g = cooperative_groups::this_grid();
  for (int r = 0; r < reps; ++r) g.sync();
  if (reps < 0 && threadIdx.x == 0) sink[blockIdx.x] = reps;  // never taken
}

extern "C" int dpf_grid_barrier_cost(int32_t ctas_per_sm, int32_t reps, double* us_per_barrier, void* stream) {
  clear_error();
  if (ctas_per_sm < 1 || reps < 1 || !us_per_barrier) return fail(DPF_E_INVALID, "dpf_grid_barrier_cost: bad argument");
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_barrier_probe, 256, 0));
  if (occ < ctas_per_sm) return fail(DPF_E_INVALID, "dpf_grid_barrier_cost: at most %d CTAs per SM fit", occ);
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = num_sms() * ctas_per_sm;
  int* sink = nullptr;
  cudaEvent_t e[4];
  for (auto& x : e) CK(cudaEventCreate(&x));
  int n0 = 0, n1 = reps;
  void* a0[] = {&n0, &sink};
  void* a1[] = {&n1, &sink};
  cudaError_t err = cudaLaunchCooperativeKernel((const void*)k_barrier_probe, grid, 256, a1, 0, s);  // warm-up
  float t0 = 0.f, t1 = 0.f;
  if (err == cudaSuccess) {
    cudaEventRecord(e[0], s);
    err = cudaLaunchCooperativeKernel((const void*)k_barrier_probe, grid, 256, a0, 0, s);
    cudaEventRecord(e[1], s);
  }
  if (err == cudaSuccess) {
    cudaEventRecord(e[2], s);
    err = cudaLaunchCooperativeKernel((const void*)k_barrier_probe, grid, 256, a1, 0, s);
    cudaEventRecord(e[3], s);
  }
  if (err == cudaSuccess) err = cudaEventSynchronize(e[3]);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t0, e[0], e[1]);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t1, e[2], e[3]);
  for (auto& x : e) cudaEventDestroy(x);
  if (err != cudaSuccess) return fail(DPF_E_CUDA, "dpf_grid_barrier_cost: %s", cudaGetErrorString(err));
  *us_per_barrier = 1e3 * (double)(t1 - t0) / reps;
  return DPF_OK;
}

extern "C" int dpf_iterations_done(const dpf_workspace* w, int32_t* n_iter) {
  if (!w || !n_iter) return fail(DPF_E_INVALID, "dpf_iterations_done: NULL argument");
  *n_iter = w->t_done;
  return DPF_OK;
}

extern "C" int dpf_solve_end(dpf_workspace* w, const dpf_batch* b, void* stream) {
  dpf::Range nvtx_range("dpf_solve_end");
  clear_error();
  if (!w || !w->begun) return fail(DPF_E_STATE, "dpf_solve_end before dpf_solve_begin");
  if (!b || b->n_case != w->K) return fail(DPF_E_INVALID, "dpf_solve_end: batch differs from dpf_solve_begin");
  cudaStream_t s = (cudaStream_t)stream;
  const dpf_ybus* y = w->y;
  const bool hio = b->host_io != 0;
  TRY(launch_check_any(w, s, true));
  const size_t E = (size_t)y->n * w->Kp;
  const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
  if (b->va || b->vm) {
    if (w->precision == DPF_FP64) {
      k_master64<double2><<<nb, 256, 0, s>>>((const double2*)w->ms, w->tmp_a, w->tmp_b, E);
    } else {
      k_master64<float4><<<nb, 256, 0, s>>>((const float4*)w->ms, w->tmp_a, w->tmp_b, E);
    }
    CKLAUNCH();
    w->launches++;
    if (b->va) TRY(to_user(w, w->tmp_a, hio, w->st_a, b->va, s));
    if (b->vm) TRY(to_user(w, w->tmp_b, hio, w->st_b, b->vm, s));
  }
  const cudaMemcpyKind kind = hio ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (b->iters) CK(cudaMemcpyAsync(b->iters, w->iters, (size_t)w->K * 4, kind, s));
  if (b->status) CK(cudaMemcpyAsync(b->status, w->status, (size_t)w->K * 4, kind, s));
  if (b->max_mismatch) CK(cudaMemcpyAsync(b->max_mismatch, w->out_max, (size_t)w->K * 8, kind, s));
  if (b->loss) CK(cudaMemcpyAsync(b->loss, w->out_loss, (size_t)w->K * 8, kind, s));
  if (hio) CK(cudaStreamSynchronize(s));
  w->begun = false;
  return DPF_OK;
}

static int solve_batched(const dpf_ybus* y, dpf_workspace* w, const dpf_batch* b, const dpf_solve_opts* o,
                         cudaStream_t s) {
  TRY(dpf_solve_begin(y, w, b, o, s));
  const int ce = o->check_every;
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  bool pending = false;
  int rc = DPF_OK;
  while (w->t_done < o->max_iter) {
    const int n = std::min(ce - (w->t_done % ce), o->max_iter - w->t_done);
    if ((rc = dpf_solve_iterate(w, n, s))) break;
    // non-blocking poll of the active count, one interval behind
    if (pending && cudaEventQuery(ev) == cudaSuccess) {
      pending = false;
      if (*w->h_n_active == 0) break;
    }
    if (!pending) {
      cudaMemcpyAsync(w->h_n_active, w->n_active, 4, cudaMemcpyDeviceToHost, s);
      cudaEventRecord(ev, s);
      pending = true;
    }
  }
  if (pending) cudaEventSynchronize(ev);
  cudaEventDestroy(ev);
  if (rc != DPF_OK) return rc;
  return dpf_solve_end(w, b, s);
}

// The plain form: one case at a time, one iteration per host round trip.
static int solve_plain(const dpf_ybus* y, dpf_workspace* w, const dpf_batch* b, const dpf_solve_opts* o,
                       cudaStream_t s) {
  dpf_solve_opts po = *o;
  po.check_every = 1;
  po.use_graph = 0;
  po.lanes = 1;
  const size_t N = (size_t)y->n;
  for (int k = 0; k < b->n_case; ++k) {
    dpf_batch one;
    memset(&one, 0, sizeof one);
    one.n_case = 1;
    one.host_io = b->host_io;
    auto off = [&](const double* p) { return p ? p + (size_t)k * N : nullptr; };
    one.p_spec = off(b->p_spec);
    one.q_spec = off(b->q_spec);
    one.vm_set = off(b->vm_set);
    one.outage = b->outage ? b->outage + k : nullptr;
    one.va = b->va ? b->va + (size_t)k * N : nullptr;
    one.vm = b->vm ? b->vm + (size_t)k * N : nullptr;
    one.iters = b->iters ? b->iters + k : nullptr;
    one.status = b->status ? b->status + k : nullptr;
    one.max_mismatch = b->max_mismatch ? b->max_mismatch + k : nullptr;
    one.loss = b->loss ? b->loss + k : nullptr;
    one.va_start = b->va_start;
    one.vm_start = b->vm_start;
    TRY(dpf_solve_begin(y, w, &one, &po, s));
    while (w->t_done < po.max_iter) {
      TRY(dpf_solve_iterate(w, 1, s));
      // host stop test of Alg. 1 (the FP64 test runs at the start of each iteration)
      int32_t act = 0;
      TRY(dpf_active_count(w, &act, s));
      if (act == 0) break;
    }
    TRY(dpf_solve_end(w, &one, s));
  }
  return DPF_OK;
}

extern "C" int dpf_solve_batch(const dpf_ybus* y, dpf_workspace* ws, const dpf_batch* b,
                               const dpf_solve_opts* o, void* stream) {
  dpf::Range nvtx_range("dpf_solve_batch");
  clear_error();
  if (!y || !b || !o) return fail(DPF_E_INVALID, "dpf_solve_batch: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  dpf_workspace* w = ws;
  if (!w) TRY(dpf_workspace_create(y, b->n_case, &w));
  const int rc = o->plain ? solve_plain(y, w, b, o, s) : solve_batched(y, w, b, o, s);
  if (!ws) {
    cudaStreamSynchronize(s);
    dpf_workspace_free(w);
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Adam on a parameter vector (parameter identification)
// ---------------------------------------------------------------------------
__global__ void k_adam_params(int n, double* __restrict__ x, const double* __restrict__ g, double* __restrict__ m,
                              double* __restrict__ v, const double* __restrict__ lr_scale, double lr, double b1,
                              double b2, double eps, double bc1, double bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  const double mi = b1 * m[i] + (1.0 - b1) * gi;
  const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const double step = lr * (lr_scale ? lr_scale[i] : 1.0);
  x[i] -= step * (mi / bc1) / (sqrt(vi / bc2) + eps);
}

extern "C" int dpf_adam_update(int32_t n, double* x, const double* grad, double* m, double* v,
                               const double* lr_scale, int32_t t, double lr, double beta1, double beta2, double eps,
                               void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!x || !grad || !m || !v))) return fail(DPF_E_INVALID, "dpf_adam_update: bad arguments");
  if (t < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps >= 0))
    return fail(DPF_E_INVALID, "dpf_adam_update: invalid step or hyper-parameters");
  if (n == 0) return DPF_OK;
  double b1t = 1.0, b2t = 1.0;  // host powers: one scalar each per call
  for (int k = 0; k < t; ++k) { b1t *= beta1; b2t *= beta2; }
  k_adam_params<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, x, grad, m, v, lr_scale, lr, beta1, beta2,
                                                                    eps, 1.0 - b1t, 1.0 - b2t);
  CKLAUNCH();
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: launch shape of the solve loop, timed on the caller's batch
// ---------------------------------------------------------------------------
extern "C" int dpf_autotune(const dpf_ybus* y, dpf_workspace* w, const dpf_batch* b, dpf_solve_opts* o,
                            int32_t iters, void* stream) {
  dpf::Range nvtx_range("dpf_autotune");
  clear_error();
  if (!y || !w || !b || !o) return fail(DPF_E_INVALID, "dpf_autotune: NULL argument");
  if (iters < 1) return fail(DPF_E_INVALID, "iters must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<long long> key = {b->n_case, o->precision, (long long)y->n, y->nnz, b->outage != nullptr,
                                      b->p_spec != nullptr};
  for (auto& kv : w->tune_cache)
    if (kv.first == key) {
      o->lanes = kv.second[0];
      o->warps = kv.second[1];
      o->row_blocks = kv.second[2];
      o->pair_cases = kv.second[3];
      o->stage_v = kv.second[4];
      o->stage_y = kv.second[5];
      return DPF_OK;
    }
  const int K = b->n_case;
  const int auto_lanes = std::min(32, pow2ceil(K));
  std::vector<int> lanes_c = {auto_lanes};
  if (auto_lanes >= 8) { lanes_c.push_back(auto_lanes / 2); lanes_c.push_back(auto_lanes / 4); }
  std::vector<int> pair_c = {0};
  if ((o->precision == DPF_FP32 || o->precision == DPF_FP32R) && K >= 64) pair_c = {0, 1, 2, 3};
  // row blocks: the automatic choice and multiples of it
  dpf_solve_opts base = *o;
  base.max_iter = 2 * iters + 4 * std::max(1, o->check_every) + 8;
  base.lanes = auto_lanes;
  base.warps = 8;
  base.row_blocks = 0;
  base.pair_cases = 0;
  base.stage_v = 0;
  base.stage_y = 0;
  choose_shape(w, &base, K);
  // single-case FP32 solves: global-memory or staged Y rows
  std::vector<int> sy_c = {0};
  if (auto_lanes == 1 && (o->precision == DPF_FP32 || o->precision == DPF_FP32R)) sy_c = {0, 1};
  const int gy_auto = w->gy;
  std::vector<int> rb_c = {0, gy_auto, 2 * gy_auto, 4 * gy_auto};  // 0: wave-aligned automatic choice
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  dpf_solve_opts best = base;
  int rc = DPF_OK;
  for (int ln : lanes_c)
    for (int pc : pair_c)
      for (int wp : {4, 8})
        for (int rb : rb_c)
          for (int sv : {0, 1})
            for (int sy : sy_c) {
          if (pc && ln != 32) continue;
          if (sv && ln != 32) continue;
          dpf_solve_opts c = base;
          c.lanes = ln;
          c.pair_cases = pc;
          c.warps = wp;
          c.row_blocks = rb;
          c.stage_v = sv;
          c.stage_y = sy;
          if ((rc = dpf_solve_begin(y, w, b, &c, s)) != DPF_OK) break;
          const int ce = std::max(1, c.check_every);
          if ((rc = dpf_solve_iterate(w, ce, s)) != DPF_OK) break;  // warm-up, builds the graph
          cudaEventRecord(e0, s);
          const int n = (iters + ce - 1) / ce * ce;
          if ((rc = dpf_solve_iterate(w, n, s)) != DPF_OK) break;
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= n;
          if (ms < best_ms) {
            best_ms = ms;
            best = c;
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  w->begun = false;
  ws_drop_graph(w);
  if (rc != DPF_OK) return rc;
  o->lanes = best.lanes;
  o->warps = best.warps;
  o->row_blocks = best.row_blocks;
  o->pair_cases = best.pair_cases;
  o->stage_v = best.stage_v;
  o->stage_y = best.stage_y;
  w->tune_cache.push_back({key, {best.lanes, best.warps, best.row_blocks, best.pair_cases, best.stage_v,
                                 best.stage_y}});
  return DPF_OK;
}

// ---------------------------------------------------------------------------
// Evaluation entry points
// ---------------------------------------------------------------------------
static int eval_setup(const dpf_ybus* y, dpf_workspace* w, int K, int precision, const double* va,
                      const double* vm, const double* p, const double* q, const int32_t* outage,
                      cudaStream_t s) {
  TRY(common_checks(y, w, K));
  if (precision != DPF_FP32 && precision != DPF_FP64) return fail(DPF_E_INVALID, "unknown precision");
  if (!va || !vm) return fail(DPF_E_INVALID, "va and vm are required");
  w->begun = false;
  w->pid_ready = false;
  ws_drop_graph(w);
  dpf_default_opts(&w->opts);
  w->opts.precision = precision;
  w->precision = precision;
  w->K = K;
  choose_shape(w, nullptr, K);
  TRY(upload_windows(w, s));
  TRY(precision == DPF_FP64 ? set_smem_attr<double>(std::max(w->smem, w->ysmem_b))
                            : set_smem_attr<float>(std::max(w->smem, w->ysmem_b)));
  TRY(ws_reserve(w, w->Kp, 0));
  StateIn in;
  memset(&in, 0, sizeof in);
  in.K = K;
  in.va = va;
  in.vm = vm;
  in.p = p;
  in.q = q;
  in.outage = outage;
  return precision == DPF_FP64 ? init_state<double>(w, in, s) : init_state<float>(w, in, s);
}

template <class R>
static int power_impl(dpf_workspace* w, double* p_calc, double* q_calc, cudaStream_t s) {
  Plan<R> P = make_plan<R>(w);
  P.it.sbuf = (typename Prec<R>::C*)w->sbuf;
  P.it.loss_part = nullptr;
  P.it.n_active = nullptr;
  P.it.tile_cnt = nullptr;
  k_fwd<R><<<P.grid, P.block, P.smem, s>>>(P.it);
  w->launches++;
  const size_t E = (size_t)w->y->n * w->Kp;
  const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
  k_widen<R><<<nb, 256, 0, s>>>((const R*)w->sbuf, w->tmp_a, E, 2, 1.0);
  w->launches++;
  k_widen<R><<<nb, 256, 0, s>>>((const R*)w->sbuf + 1, w->tmp_b, E, 2, 1.0);
  w->launches++;
  CKLAUNCH();
  if (p_calc) TRY(to_user(w, w->tmp_a, false, nullptr, p_calc, s));
  if (q_calc) TRY(to_user(w, w->tmp_b, false, nullptr, q_calc, s));
  return DPF_OK;
}

extern "C" int dpf_power(const dpf_ybus* y, dpf_workspace* w, int32_t n_case, const double* va,
                         const double* vm, const int32_t* outage, int32_t precision, double* p_calc,
                         double* q_calc, void* stream) {
  dpf::Range nvtx_range("dpf_power");
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  TRY(eval_setup(y, w, n_case, precision, va, vm, nullptr, nullptr, outage, s));
  return precision == DPF_FP64 ? power_impl<double>(w, p_calc, q_calc, s) : power_impl<float>(w, p_calc, q_calc, s);
}

// dL/d(series g, b, b_ch) of every branch, summed over the cases, from w and V
// (branch adjoint; written into zeroed outputs).
template <class R>
static int launch_edge_grad(dpf_workspace* w, double* d_g, double* d_b, double* d_bch, cudaStream_t s) {
  using C = typename Prec<R>::C;
  const dpf_ybus* y = w->y;
  if (d_g) CK(cudaMemsetAsync(d_g, 0, (size_t)y->m * 8, s));
  if (d_b) CK(cudaMemsetAsync(d_b, 0, (size_t)y->m * 8, s));
  if (d_bch) CK(cudaMemsetAsync(d_bch, 0, (size_t)y->m * 8, s));
  EdgeArgs<R> ea;
  memset(&ea, 0, sizeof ea);
  ea.M = y->m;
  ea.K = w->K;
  ea.Kp = w->Kp;
  ea.lanes = w->lanes;
  ea.br_f = y->dev.br_f;
  ea.br_t = y->dev.br_t;
  ea.itap = y->dev.br_itap;
  ea.V = (const C*)w->V;
  ea.W = (const C*)w->W;
  ea.d_g = d_g;
  ea.d_b = d_b;
  ea.d_bch = d_bch;
  const int rpw = 32 / w->lanes;
  const int gy = std::max(1, std::min((y->m + w->warps * rpw - 1) / (w->warps * rpw), 65535));
  k_edge_grad<R><<<dim3(w->gx, gy), dim3(w->warps * 32), 0, s>>>(ea);
  w->launches++;
  CKLAUNCH();
  return DPF_OK;
}

template <class R>
static int loss_backward_impl(dpf_workspace* w, double* loss, double* d_va, double* d_vm, double* d_p,
                              double* d_q, double* d_g, double* d_b, double* d_bch, cudaStream_t s) {
  using C = typename Prec<R>::C;
  const dpf_ybus* y = w->y;
  Plan<R> P = make_plan<R>(w);
  P.it.cbuf = (d_p || d_q) ? (C*)w->cbuf : nullptr;
  P.it.loss_part = nullptr;  // (the loss is the FP64 pass's)
  P.it.mx32 = nullptr;
  P.it.n_active = nullptr;
  P.it.tile_cnt = nullptr;
  k_fwd<R><<<P.grid, P.block, P.smem, s>>>(P.it);
  w->launches++;
  CKLAUNCH();
  const size_t E = (size_t)y->n * w->Kp;
  const int nb = (int)std::min<size_t>((E + 255) / 256, (size_t)num_sms() * 16);
  if (d_va || d_vm) {  // the voltage adjoint (the branch adjoint needs only w and V)
    P.it.gva = (R*)w->tmp_c;  // gradient scratch: [N][Kp] R each
    P.it.gvm = (R*)w->sbuf;
    P.itb = P.it;
    P.itb.rpb = w->rpb_b;
    k_adj<R><<<P.gridb, P.block, P.ysmem, s>>>(P.itb);
    w->launches++;
    CKLAUNCH();
  }
  if (d_va) {
    k_widen<R><<<nb, 256, 0, s>>>((const R*)w->tmp_c, w->tmp_a, E, 1, 1.0);
    w->launches++;
    CKLAUNCH();
    TRY(to_user(w, w->tmp_a, false, nullptr, d_va, s));
  }
  if (d_vm) {
    k_widen<R><<<nb, 256, 0, s>>>((const R*)w->sbuf, w->tmp_a, E, 1, 1.0);
    w->launches++;
    CKLAUNCH();
    TRY(to_user(w, w->tmp_a, false, nullptr, d_vm, s));
  }
  if (d_p) {
    k_widen<R><<<nb, 256, 0, s>>>((const R*)w->cbuf, w->tmp_a, E, 2, -1.0);
    w->launches++;
    CKLAUNCH();
    TRY(to_user(w, w->tmp_a, false, nullptr, d_p, s));
  }
  if (d_q) {
    k_widen<R><<<nb, 256, 0, s>>>((const R*)w->cbuf + 1, w->tmp_a, E, 2, -1.0);
    w->launches++;
    CKLAUNCH();
    TRY(to_user(w, w->tmp_a, false, nullptr, d_q, s));
  }
  if (d_g || d_b || d_bch) TRY(launch_edge_grad<R>(w, d_g, d_b, d_bch, s));
  if (loss) {
    TRY(launch_check<R>(w, s, true));
    CK(cudaMemcpyAsync(loss, w->out_loss, (size_t)w->K * 8, cudaMemcpyDeviceToDevice, s));
  }
  return DPF_OK;
}

// Y_bus values from caller series admittances (the workspace's local copy).
static void rebuild_local_y(const dpf_ybus* y, dpf_workspace* w, const double* g_series, const double* b_series,
                            cudaStream_t s) {
  YValArgs ya;
  ya.N = y->n;
  ya.rp = y->dev.row_ptr;
  ya.col = y->dev.col;
  ya.ebr = y->dev.ebr;
  ya.br_f = y->dev.br_f;
  ya.g = g_series;
  ya.b = b_series;
  ya.bch = y->dev.br_bch;
  ya.itap = y->dev.br_itap;
  ya.ent32 = w->ent_loc;
  ya.val64 = w->val_loc;
  k_ybus_values<<<(y->n + 127) / 128, 128, 0, s>>>(ya);
  w->use_local_y = true;
}

extern "C" int dpf_loss_backward(const dpf_ybus* y, dpf_workspace* w, int32_t n_case, const double* va,
                                 const double* vm, const double* p_spec, const double* q_spec,
                                 const int32_t* outage, const double* g_series, const double* b_series,
                                 int32_t precision, double* loss, double* d_va, double* d_vm, double* d_p,
                                 double* d_q, double* d_g, double* d_b, double* d_bch, void* stream) {
  dpf::Range nvtx_range("dpf_loss_backward");
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if ((g_series == nullptr) != (b_series == nullptr))
    return fail(DPF_E_INVALID, "g_series and b_series must be given together");
  TRY(eval_setup(y, w, n_case, precision, va, vm, p_spec, q_spec, outage, s));
  if (g_series) {
    rebuild_local_y(y, w, g_series, b_series, s);
    CKLAUNCH();
  }
  const int rc = precision == DPF_FP64
                     ? loss_backward_impl<double>(w, loss, d_va, d_vm, d_p, d_q, d_g, d_b, d_bch, s)
                     : loss_backward_impl<float>(w, loss, d_va, d_vm, d_p, d_q, d_g, d_b, d_bch, s);
  w->use_local_y = false;
  return rc;
}

// ---------------------------------------------------------------------------
// Parameter identification: operating points staged once, then per step the
// Y values from (g, b), the forward pass and the branch adjoint.
// ---------------------------------------------------------------------------
extern "C" int dpf_paramid_begin(const dpf_ybus* y, dpf_workspace* w, int32_t n_case, const double* va,
                                 const double* vm, const double* p_spec, const double* q_spec, int32_t precision,
                                 void* stream) {
  dpf::Range nvtx_range("dpf_paramid_begin");
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  TRY(eval_setup(y, w, n_case, precision, va, vm, p_spec, q_spec, nullptr, s));
  w->pid_ready = true;
  return DPF_OK;
}

template <class R>
static int paramid_impl(dpf_workspace* w, double* d_g, double* d_b, double* d_bch, double* loss, cudaStream_t s) {
  k_activate<<<(w->Kp + 255) / 256, 256, 0, s>>>(w->active, w->K, w->Kp);
  w->launches++;
  Plan<R> P = make_plan<R>(w);
  P.it.cbuf = nullptr;
  P.it.loss_part = nullptr;
  P.it.mx32 = nullptr;
  P.it.n_active = nullptr;
  P.it.tile_cnt = nullptr;
  k_fwd<R><<<P.grid, P.block, P.smem, s>>>(P.it);  // w = c conj(V) at the staged points (V unchanged)
  w->launches++;
  CKLAUNCH();
  if (d_g || d_b || d_bch) TRY(launch_edge_grad<R>(w, d_g, d_b, d_bch, s));
  if (loss) {
    TRY(launch_check<R>(w, s, true));
    CK(cudaMemcpyAsync(loss, w->out_loss, (size_t)w->K * 8, cudaMemcpyDeviceToDevice, s));
  }
  return DPF_OK;
}

extern "C" int dpf_paramid_step(const dpf_ybus* y, dpf_workspace* w, const double* g_series,
                                const double* b_series, double* d_g, double* d_b, double* d_bch, double* loss,
                                void* stream) {
  dpf::Range nvtx_range("dpf_paramid_step");
  clear_error();
  if (!y || !w) return fail(DPF_E_INVALID, "dpf_paramid_step: NULL handle");
  if (w->y != y) return fail(DPF_E_INVALID, "workspace was created for another Y_bus");
  if (!w->pid_ready) return fail(DPF_E_STATE, "dpf_paramid_step: no operating points staged (dpf_paramid_begin)");
  if (!g_series || !b_series) return fail(DPF_E_INVALID, "dpf_paramid_step: g_series and b_series are required");
  cudaStream_t s = (cudaStream_t)stream;
  rebuild_local_y(y, w, g_series, b_series, s);
  CKLAUNCH();
  const int rc = w->precision == DPF_FP64 ? paramid_impl<double>(w, d_g, d_b, d_bch, loss, s)
                                          : paramid_impl<float>(w, d_g, d_b, d_bch, loss, s);
  w->use_local_y = false;
  return rc;
}
