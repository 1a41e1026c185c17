// Batched Newton-Raphson power flow (Alg. 2) on the GPU, for the same batches
// dpf_solve_batch takes (one Y_bus, per-case injections and one outage each):
// the comparison solver of the paper and the second half of a hybrid in which
// Alg. 1 supplies the starting point (Sec. 5.4, Sec. 6).
//
// Per Newton iteration, for every case still iterating:
//   k_nr_volt      V = |V| e^{j theta} (FP64)
//   k_nr_eval      I = Y' V, S = V conj(I), f, right-hand side -f (FP64)
//   k_nr_partial   per case and chunk of rows: partial max |f| and ||f||^2
//   k_nr_check     per case max |f|, loss, stop test (the host reads the
//                  number of cases left)
//   k_nr_assemble  the 2x2 Jacobian blocks of Alg. 2 on the filled pattern
//   k_nr_lu        block LU, left-looking, level by level of the elimination
//                  tree, with the forward substitution L y = -f folded into
//                  the same level pass, then U dx = y back down the tree; one
//                  CTA per tile of cases, which syncs only its own threads:
//                  the cases are independent, so no CTA waits for another
//   k_nr_update    theta += dx_theta (pv, pq), |V| += dx_|V| (pq)
// The factor and the triangular solves run in the factor precision (FP64, or
// FP32: GB300 issues FP32 FMA at many times its FP64 rate, and a Newton step
// solved to FP32 accuracy still converges, linearly at a rate of about
// cond(J) 2^-24 once quadratic convergence has run out); the mismatch, the
// stop test and the state are FP64 in both.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dpf_internal.h"
#include "dpf_nr.h"

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

#define TRY(x)                   \
  do {                           \
    int s_ = (x);                \
    if (s_ != DPF_OK) return s_; \
  } while (0)

namespace {

constexpr uint8_t NR_PQ = 0, NR_SLACK = 2;  // bus types (pv = 1)
constexpr int NR_THREADS = 256;
constexpr int NR_SMEM_THREADS = 1024;
constexpr int NR_CHUNKS = 16;  // row chunks of the per-case reduction

// 2x2 block: rows (P, Q), columns (theta, |V|), row-major.
template <class T>
struct alignas(4 * sizeof(T)) Blk {
  T a, b, c, d;
};

template <class T>
__device__ __forceinline__ Blk<T> ldb(const Blk<T>* p) {
  return *p;
}
template <>
__device__ __forceinline__ Blk<double> ldb(const Blk<double>* p) {
  const double2 u = reinterpret_cast<const double2*>(p)[0], v = reinterpret_cast<const double2*>(p)[1];
  return Blk<double>{u.x, u.y, v.x, v.y};
}
template <class T>
__device__ __forceinline__ void stb(Blk<T>* p, const Blk<T>& v) {
  *p = v;
}
template <>
__device__ __forceinline__ void stb(Blk<double>* p, const Blk<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.a, v.b);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.c, v.d);
}

// acc -= x y
template <class T>
__device__ __forceinline__ void msub(Blk<T>& acc, const Blk<T>& x, const Blk<T>& y) {
  acc.a = fma(-x.a, y.a, fma(-x.b, y.c, acc.a));
  acc.b = fma(-x.a, y.b, fma(-x.b, y.d, acc.b));
  acc.c = fma(-x.c, y.a, fma(-x.d, y.c, acc.c));
  acc.d = fma(-x.c, y.b, fma(-x.d, y.d, acc.d));
}
template <class T>
__device__ __forceinline__ Blk<T> mul(const Blk<T>& x, const Blk<T>& y) {
  return Blk<T>{fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c),
                fma(x.c, y.b, x.d * y.d)};
}
// inverse of a 2x2 block; false if it is singular (or not finite)
template <class T>
__device__ __forceinline__ bool inv2(const Blk<T>& m, Blk<T>& r) {
  const T det = fma(m.a, m.d, -m.b * m.c);
  const T id = T(1) / det;
  r = Blk<T>{m.d * id, -m.b * id, -m.c * id, m.a * id};
  return det != T(0) && isfinite(id);
}

__device__ __forceinline__ double2 cmul(double2 x, double2 y) {
  return make_double2(fma(x.x, y.x, -x.y * y.y), fma(x.x, y.y, x.y * y.x));
}
__device__ __forceinline__ double2 cconj(double2 x) { return make_double2(x.x, -x.y); }
__device__ __forceinline__ double2 csub(double2 x, double2 y) { return make_double2(x.x - y.x, x.y - y.y); }

struct NrArgs {
  int N, K, Kp, C;
  double va_slack, tol, inv_m;
  int max_iter;
  // grid (device, internal order)
  const int32_t* rp;
  const int32_t* ycol;
  const double2* yval;
  const uint8_t* type;
  const double* p64;
  const double* q64;
  const double* vmset;
  const int32_t* perm;
  // schedule
  const int32_t* order;
  const int32_t* rank;
  const int32_t* frp;
  const int32_t* fcol;
  const int32_t* fdiag;
  const int32_t* ymap;
  int n_levels;
  const int32_t* lvl_ptr;
  const int4* targets;
  const int2* pairs;
  const int32_t* rlvl_ptr;
  const int4* rows;
  int64_t npos;
  // state [N][Kp]
  double* th;
  double* vm;
  double2* V;
  double2* U;    // e^{j theta}: V = |V| U
  double2* I;
  double2* X;    // right-hand side / solution, by elimination step
  double* Ps;    // per-case specification or NULL
  double* Qs;
  void* F;       // [npos][Kp] blocks
  void* Dinv;    // [N][Kp] blocks
  // per case
  int32_t* of;
  int32_t* ot;
  double2* yff;
  double2* yft;
  double2* ytt;
  int32_t* active;
  int32_t* status;
  int32_t* iters;
  int32_t* bad;
  double* maxmis;
  double* loss;
  int32_t* n_active;
  double* pmax;  // [NR_CHUNKS][Kp] partials of the stop test
  double* psum;
  double* maxmis0;  // per case: max |f| and loss of the start
  double* loss0;
  int first;        // this evaluation is of the start
};

// Per case: outage data (pi-model block of the removed branch), state flags.
__global__ void k_nr_init(NrArgs a, const int32_t* __restrict__ outage, const int32_t* __restrict__ br_f,
                          const int32_t* __restrict__ br_t, const double* __restrict__ br_r,
                          const double* __restrict__ br_x, const double* __restrict__ br_bch,
                          const double* __restrict__ br_tap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.Kp) return;
  a.active[k] = k < a.K ? 1 : 0;
  a.status[k] = DPF_CASE_MAX_ITER;
  a.iters[k] = 0;
  a.bad[k] = 0;
  a.maxmis[k] = 0.0;
  a.loss[k] = 0.0;
  const int ell = (k < a.K && outage) ? outage[k] : -1;
  if (ell < 0) {
    a.of[k] = -1;
    a.ot[k] = -1;
    return;
  }
  const double r = br_r[ell], x = br_x[ell], bch = br_bch[ell];
  const double tau = br_tap[ell] == 0.0 ? 1.0 : br_tap[ell];
  const double d = r * r + x * x, gs = r / d, bs = -x / d, t2 = tau * tau;
  a.of[k] = br_f[ell];
  a.ot[k] = br_t[ell];
  a.yff[k] = make_double2(gs / t2, (bs + 0.5 * bch) / t2);
  a.yft[k] = make_double2(-gs / tau, -bs / tau);
  a.ytt[k] = make_double2(gs, bs + 0.5 * bch);
}

// Inputs to the internal layout: start (flat or given, set-points enforced)
// and per-case specifications.
__global__ void k_nr_in(NrArgs a, const double* __restrict__ va_in, const double* __restrict__ vm_in,
                        const double* __restrict__ p_in, const double* __restrict__ q_in,
                        const double* __restrict__ vs_in, int flat) {
  const size_t n = (size_t)a.N * a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.Kp), k = (int)(e % a.Kp);
    const uint8_t t = __ldg(a.type + i);
    double th = 0.0, vm = 1.0;
    if (k < a.K) {
      const size_t u = (size_t)k * a.N + __ldg(a.perm + i);
      const double vs = vs_in ? vs_in[u] : __ldg(a.vmset + i);
      if (a.Ps) {
        a.Ps[e] = p_in[u];
        a.Qs[e] = q_in[u];
      }
      if (!flat) {
        th = va_in[u];
        vm = vm_in[u];
      }
      if (t == NR_SLACK) th = a.va_slack;
      if (t != NR_PQ) vm = vs;
    }
    a.th[e] = th;
    a.vm[e] = vm;
  }
}

__global__ void k_nr_volt(NrArgs a) {
  const size_t n = (size_t)a.N * a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    if (!a.active[e % a.Kp]) continue;
    double s, c;
    sincos(a.th[e], &s, &c);
    a.U[e] = make_double2(c, s);
    a.V[e] = make_double2(a.vm[e] * c, a.vm[e] * s);
  }
}

// Currents, power, mismatch f = [P_calc - P (pv, pq); Q_calc - Q (pq)] and
// the right-hand side -f by elimination step (0 for the identity rows).
__global__ void k_nr_eval(NrArgs a) {
  const size_t n = (size_t)a.N * a.Kp, Kp = a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Kp), k = (int)(e % Kp);
    if (!a.active[k]) continue;
    double2 cur = make_double2(0.0, 0.0);
    const int p1 = __ldg(a.rp + i + 1);
    for (int p = __ldg(a.rp + i); p < p1; ++p) {
      const double2 y = __ldg(a.yval + p), v = a.V[(size_t)__ldg(a.ycol + p) * Kp + k];
      cur.x = fma(y.x, v.x, fma(-y.y, v.y, cur.x));
      cur.y = fma(y.x, v.y, fma(y.y, v.x, cur.y));
    }
    const int of = a.of[k], ot = a.ot[k];
    if (i == of || i == ot) {  // the outaged branch's share leaves Y_bus
      const double2 vf = a.V[(size_t)of * Kp + k], vt = a.V[(size_t)ot * Kp + k];
      const double2 d = (i == of) ? cmul(a.yff[k], vf) : cmul(a.yft[k], vf);
      const double2 d2 = (i == of) ? cmul(a.yft[k], vt) : cmul(a.ytt[k], vt);
      cur = csub(csub(cur, d), d2);
    }
    const double2 v = a.V[e];
    const double2 s = cmul(v, cconj(cur));
    const uint8_t t = __ldg(a.type + i);
    const double ps = a.Ps ? a.Ps[e] : __ldg(a.p64 + i), qs = a.Ps ? a.Qs[e] : __ldg(a.q64 + i);
    const double fp = (t != NR_SLACK) ? s.x - ps : 0.0;
    const double fq = (t == NR_PQ) ? s.y - qs : 0.0;
    a.I[e] = cur;
    a.X[(size_t)__ldg(a.rank + i) * Kp + k] = make_double2(-fp, -fq);
  }
}

// Per case and chunk of rows (32 cases x 8 row groups per CTA, fixed
// summation order): partial max |f| (NaN if any entry is NaN) and partial
// ||f||^2 from the right-hand side -f.
__global__ void __launch_bounds__(256) k_nr_partial(NrArgs a) {
  __shared__ double smax[8][32], ssum[8][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int k = blockIdx.x * 32 + lane;
  const bool on = k < a.K && a.active[k];
  const int rpc = (a.N + NR_CHUNKS - 1) / NR_CHUNKS;
  const int r0 = blockIdx.y * rpc, r1 = min(a.N, r0 + rpc);
  double mx = 0.0, sm = 0.0;
  bool nan = false;
  if (on)
    for (int r = r0 + g; r < r1; r += 8) {
      const double2 x = a.X[(size_t)r * a.Kp + k];
      nan = nan || !(x.x == x.x) || !(x.y == x.y);
      mx = fmax(mx, fmax(fabs(x.x), fabs(x.y)));
      sm = fma(x.x, x.x, fma(x.y, x.y, sm));
    }
  smax[g][lane] = nan ? __longlong_as_double(0x7ff8000000000000LL) : mx;
  ssum[g][lane] = sm;
  __syncthreads();
  if (g != 0 || !on) return;
  mx = 0.0;
  sm = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double m = smax[q][lane];
    nan = nan || !(m == m);
    mx = fmax(mx, m);
    sm += ssum[q][lane];
  }
  a.pmax[(size_t)blockIdx.y * a.Kp + k] = nan ? __longlong_as_double(0x7ff8000000000000LL) : mx;
  a.psum[(size_t)blockIdx.y * a.Kp + k] = sm;
}

// Per case: max |f|, loss (1/m) ||f||^2 from the chunks' partials (fixed
// order) and the stop test of Alg. 2.
__global__ void k_nr_check(NrArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K || !a.active[k]) return;
  double mx = 0.0, sm = 0.0;
  bool nan = false;
  for (int c = 0; c < NR_CHUNKS; ++c) {
    const double m = a.pmax[(size_t)c * a.Kp + k];
    nan = nan || !(m == m);
    mx = fmax(mx, m);
    sm += a.psum[(size_t)c * a.Kp + k];
  }
  if (nan) mx = __longlong_as_double(0x7ff8000000000000LL);
  a.maxmis[k] = mx;
  a.loss[k] = sm * a.inv_m;
  if (a.first) {
    a.maxmis0[k] = mx;
    a.loss0[k] = sm * a.inv_m;
  }
  if (a.bad[k] || nan || isinf(mx)) {
    a.status[k] = DPF_CASE_DIVERGED;
    a.active[k] = 0;
  } else if (mx <= a.tol) {
    a.status[k] = DPF_CASE_CONVERGED;
    a.active[k] = 0;
  } else if (a.iters[k] >= a.max_iter) {
    a.status[k] = DPF_CASE_MAX_ITER;
    a.active[k] = 0;
  } else {
    a.iters[k] += 1;  // a Newton step follows
    atomicAdd(a.n_active, 1);
  }
}

// Jacobian blocks (Alg. 2) at every position of the filled pattern, with
// u = e^{j theta} (so V = |V| u) and W = V_i conj(Y'_ij u_j):
//   i != j: dS_i/dtheta_j = -j |V|_j W,        dS_i/d|V|_j = W
//   i == j: dS_i/dtheta_i = j (S_i - |V|_i W), dS_i/d|V|_i = u_i conj(I_i) + W
// (the element rules of Alg. 2 with T = V_i conj(Y'_ij V_j) = |V|_j W; the
// division by |V|_j cancels, and none is left: an FP64 divide costs many
// issue slots here).  Computed in the factor's precision T (the FP64 state
// rounded once); rows P = Re, Q = Im; equations and unknowns Alg. 2 leaves
// out are zeroed, with a 1 on the diagonal.  Fill positions start at 0.  One
// thread per (block row, case) walks the row's positions.
template <class T>
struct Cx {
  T x, y;
};
template <class T>
__device__ __forceinline__ Cx<T> cx(double2 v) {
  return Cx<T>{(T)v.x, (T)v.y};
}
template <class T>
__device__ __forceinline__ Cx<T> mulc(Cx<T> a, Cx<T> b) {  // a conj(b)
  return Cx<T>{fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y)};
}
template <class T>
__device__ __forceinline__ Cx<T> mul(Cx<T> a, Cx<T> b) {
  return Cx<T>{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}

// One block row of case k: its positions' blocks to dst[q * stride].
template <class T>
__device__ __forceinline__ void assemble_row(const NrArgs& a, int r, int k, Blk<T>* __restrict__ dst, size_t stride) {
  const size_t Kp = a.Kp;
  const double2* __restrict__ U = a.U;
  const double* __restrict__ VM = a.vm;
  const int i = __ldg(a.order + r);
  const size_t ei = (size_t)i * Kp + k;
  const Cx<T> vi = cx<T>(a.V[ei]), ii = cx<T>(a.I[ei]);
  const Cx<T> si = mulc(vi, ii);             // S_i
  const Cx<T> sdi = mulc(cx<T>(U[ei]), ii);  // S_i / |V|_i
  const uint8_t ti = __ldg(a.type + i);
  const bool rp = ti != NR_SLACK, rq = ti == NR_PQ;
  const int of = a.of[k], ot = a.ot[k];
  const int q1 = __ldg(a.frp + r + 1);
  for (int q = __ldg(a.frp + r); q < q1; ++q) {
    const int j = __ldg(a.order + __ldg(a.fcol + q));
    const int yp = __ldg(a.ymap + q);
    Blk<T> b{T(0), T(0), T(0), T(0)};
    if (yp >= 0) {
      double2 y = __ldg(a.yval + yp);
      if (of >= 0) {
        if (i == of && j == of) y = csub(y, a.yff[k]);
        else if (i == ot && j == ot) y = csub(y, a.ytt[k]);
        else if ((i == of && j == ot) || (i == ot && j == of)) y = csub(y, a.yft[k]);
      }
      const size_t ej = (size_t)j * Kp + k;
      const Cx<T> w = mulc(vi, mul(cx<T>(y), cx<T>(U[ej])));
      const T vmj = (T)VM[ej];
      T ba, bb, bc, bd;
      if (i != j) {
        ba = vmj * w.y;
        bc = -vmj * w.x;
        bb = w.x;
        bd = w.y;
      } else {
        ba = fma(vmj, w.y, -si.y);
        bc = fma(-vmj, w.x, si.x);
        bb = sdi.x + w.x;
        bd = sdi.y + w.y;
      }
      const uint8_t tj = __ldg(a.type + j);
      const bool ct = tj != NR_SLACK, cv = tj == NR_PQ;
      b.a = (rp && ct) ? ba : T(0);
      b.b = (rp && cv) ? bb : T(0);
      b.c = (rq && ct) ? bc : T(0);
      b.d = (rq && cv) ? bd : T(0);
      if (i == j) {
        if (!rp) b.a = T(1);
        if (!rq) b.d = T(1);
      }
    }
    stb(dst + (size_t)q * stride, b);
  }
}

template <class T>
__global__ void k_nr_assemble(NrArgs a) {
  Blk<T>* F = static_cast<Blk<T>*>(a.F);
  const size_t n = (size_t)a.N * a.Kp, Kp = a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Kp), k = (int)(e % Kp);
    if (a.active[k]) assemble_row(a, r, k, F + k, Kp);
  }
}

// Right-hand side / solution entries: FP64 pairs in global memory, pairs of
// the factor's type in shared memory.
template <class T>
__device__ __forceinline__ Cx<T> ldx(const double2* p) {
  const double2 v = *p;
  return Cx<T>{(T)v.x, (T)v.y};
}
template <class T>
__device__ __forceinline__ Cx<T> ldx(const Cx<T>* p) {
  return *p;
}
template <class T>
__device__ __forceinline__ void stx(double2* p, Cx<T> v) {
  *p = make_double2((double)v.x, (double)v.y);
}
template <class T>
__device__ __forceinline__ void stx(Cx<T>* p, Cx<T> v) {
  *p = v;
}

// acc minus the updates of one target: sum over its pairs of L(i,k) U(k,j)
template <class T>
__device__ __forceinline__ void apply_pairs(Blk<T>& acc, const Blk<T>* F, size_t fs, const int2* __restrict__ pairs,
                                            int p, int p1) {
  for (; p + 1 < p1; p += 2) {
    const int2 q0 = __ldg(pairs + p), q1 = __ldg(pairs + p + 1);
    const Blk<T> l0 = ldb(F + (size_t)q0.x * fs), u0 = ldb(F + (size_t)q0.y * fs);
    const Blk<T> l1 = ldb(F + (size_t)q1.x * fs), u1 = ldb(F + (size_t)q1.y * fs);
    msub(acc, l0, u0);
    msub(acc, l1, u1);
  }
  if (p < p1) {
    const int2 q0 = __ldg(pairs + p);
    msub(acc, ldb(F + (size_t)q0.x * fs), ldb(F + (size_t)q0.y * fs));
  }
}

// Block LU of one case and both triangular solves, in one pass per level of
// the elimination tree (leaves first) and one back down.  At level l every
// target position (i, j) whose pivot p = min(i, j) sits on level l takes
// its updates -L(i,k) U(k,j) from earlier pivots (all on lower levels, final
// after the previous level's barrier); an L position also forms its pivot's
// updated diagonal block D_p itself (a short list for this kind of grid) and
// stores L(i,p) = A(i,p) D_p^-1, so one barrier per level suffices; the
// diagonal target of row r stores D_r^-1 and the forward substitution
// y_r = b_r - sum_c L(r,c) y_c (its L columns are descendants: final).  The
// assembled diagonal blocks are only read.  Then, root first,
// x_r = D_r^-1 (y_r - sum_c U(r,c) x_c), in place in X.  Block q of the case
// is F[q * fs], the inverse diagonal of row r Dv[r * ds], its right-hand
// side X[r * xs]; this thread takes every S-th target from `slot` on.
template <class T, class XT>
__device__ __forceinline__ void lu_levels(const NrArgs& a, Blk<T>* F, size_t fs, Blk<T>* Dv, size_t ds, XT* X,
                                          size_t xs, int slot, int S, bool on, int32_t* bad) {
  for (int l = 0; l < a.n_levels; ++l) {
    const int t0 = __ldg(a.lvl_ptr + l), t1 = __ldg(a.lvl_ptr + l + 1);
    int t = t0 + slot;
    int4 na, nb;  // the schedule entry of this slot's next target, fetched one step ahead
    if (on && t < t1) {
      na = __ldg(a.targets + 2 * t);
      nb = __ldg(a.targets + 2 * t + 1);
    }
    if (on)
      for (; t < t1; t += S) {
        const int4 ta = na, tb = nb;
        if (t + S < t1) {
          na = __ldg(a.targets + 2 * (t + S));
          nb = __ldg(a.targets + 2 * (t + S) + 1);
        }
        Blk<T> acc = ldb(F + (size_t)ta.x * fs);
        apply_pairs(acc, F, fs, a.pairs, ta.y, ta.z);
        if (ta.w == NR_U) {
          stb(F + (size_t)ta.x * fs, acc);
          continue;
        }
        Blk<T> d = acc;
        if (ta.w == NR_L) {
          d = ldb(F + (size_t)tb.x * fs);
          apply_pairs(d, F, fs, a.pairs, tb.y, tb.z);
        }
        Blk<T> di;
        const bool ok = inv2(d, di);
        if (ta.w == NR_L) {
          stb(F + (size_t)ta.x * fs, mul(acc, di));
          continue;
        }
        if (!ok) *bad = 1;
        const int r = tb.w;
        stb(Dv + (size_t)r * ds, di);
        Cx<T> y = ldx<T>(X + (size_t)r * xs);
        const int q1 = ta.x;  // the row's L positions (from tb.x) precede its diagonal
        for (int q = tb.x; q < q1; ++q) {
          const Blk<T> m = ldb(F + (size_t)q * fs);
          const Cx<T> x = ldx<T>(X + (size_t)__ldg(a.fcol + q) * xs);
          y.x = fma(-m.a, x.x, fma(-m.b, x.y, y.x));
          y.y = fma(-m.c, x.x, fma(-m.d, x.y, y.y));
        }
        stx(X + (size_t)r * xs, y);
      }
    __syncthreads();
  }
  for (int l = a.n_levels - 1; l >= 0; --l) {
    const int t0 = __ldg(a.rlvl_ptr + l), t1 = __ldg(a.rlvl_ptr + l + 1);
    if (on)
      for (int t = t0 + slot; t < t1; t += S) {
        const int4 rw = __ldg(a.rows + t);  // {r, first U position, end of row}
        const int r = rw.x;
        Cx<T> y = ldx<T>(X + (size_t)r * xs);
        for (int q = rw.y; q < rw.z; ++q) {
          const Blk<T> m = ldb(F + (size_t)q * fs);
          const Cx<T> x = ldx<T>(X + (size_t)__ldg(a.fcol + q) * xs);
          y.x = fma(-m.a, x.x, fma(-m.b, x.y, y.x));
          y.y = fma(-m.c, x.x, fma(-m.d, x.y, y.y));
        }
        const Blk<T> di = ldb(Dv + (size_t)r * ds);
        stx(X + (size_t)r * xs, Cx<T>{fma(di.a, y.x, di.b * y.y), fma(di.c, y.x, di.d * y.y)});
      }
    __syncthreads();
  }
}

// Global-memory form: C cases per CTA are the lanes (their blocks adjacent),
// the remaining thread index is the slot.
template <class T>
__global__ void __launch_bounds__(NR_THREADS) k_nr_lu(NrArgs a) {
  const int lane = threadIdx.x & (a.C - 1), slot = threadIdx.x / a.C, S = blockDim.x / a.C;
  const int k = blockIdx.x * a.C + lane;
  const bool on = k < a.K && a.active[k];
  if (!__syncthreads_or(on)) return;  // no case of this tile is iterating
  const size_t Kp = a.Kp;
  lu_levels(a, static_cast<Blk<T>*>(a.F) + k, Kp, static_cast<Blk<T>*>(a.Dinv) + k, Kp, a.X + k, Kp, slot, S, on,
            a.bad + k);
}

// Shared-memory form, for grids whose factor of one case fits: one CTA per
// case assembles its Jacobian straight into shared memory (the factor never
// goes to HBM), factorises and solves there, and writes dx back.
template <class T>
__global__ void __launch_bounds__(NR_SMEM_THREADS) k_nr_lu_smem(NrArgs a) {
  extern __shared__ __align__(16) unsigned char nr_smem[];
  const int k = blockIdx.x;
  if (!a.active[k]) return;  // the same for the whole CTA
  Blk<T>* Fs = reinterpret_cast<Blk<T>*>(nr_smem);
  Blk<T>* Ds = Fs + a.npos;
  Cx<T>* Xs = reinterpret_cast<Cx<T>*>(Ds + a.N);
  const size_t Kp = a.Kp;
  for (int r = threadIdx.x; r < a.N; r += blockDim.x) {
    Xs[r] = ldx<T>(a.X + (size_t)r * Kp + k);
    assemble_row(a, r, k, Fs, 1);
  }
  __syncthreads();
  lu_levels(a, Fs, 1, Ds, 1, Xs, 1, (int)threadIdx.x, (int)blockDim.x, true, a.bad + k);
  for (int r = threadIdx.x; r < a.N; r += blockDim.x) stx(a.X + (size_t)r * Kp + k, Xs[r]);
}

// Shared memory the shared-memory form needs for one case.
template <class T>
size_t lu_smem_bytes(int64_t npos, int n) {
  return (size_t)(npos + n) * sizeof(Blk<T>) + (size_t)n * sizeof(Cx<T>);
}

__global__ void k_nr_update(NrArgs a) {
  const size_t n = (size_t)a.N * a.Kp, Kp = a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Kp), k = (int)(e % Kp);
    if (!a.active[k] || a.bad[k]) continue;
    const int i = __ldg(a.order + r);
    const uint8_t t = __ldg(a.type + i);
    const double2 dx = a.X[e];
    const size_t ei = (size_t)i * Kp + k;
    if (t != NR_SLACK) a.th[ei] += dx.x;
    if (t == NR_PQ) a.vm[ei] += dx.y;
  }
}

// Solution and per-case results to the caller's arrays (case-major, user bus
// order).  With `fallback`, a case that did not converge keeps the start the
// caller passed in va/vm, and its start's max |f| and loss are reported.
__global__ void k_nr_out(NrArgs a, double* __restrict__ va, double* __restrict__ vm, int fallback) {
  const size_t n = (size_t)a.N * a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.Kp), k = (int)(e % a.Kp);
    if (k >= a.K || (fallback && a.status[k] != DPF_CASE_CONVERGED)) continue;
    const size_t u = (size_t)k * a.N + __ldg(a.perm + i);
    va[u] = a.th[e];
    vm[u] = a.vm[e];
  }
}

__global__ void k_nr_case_out(NrArgs a, int32_t* iters, int32_t* status, double* maxmis, double* loss,
                              int fallback) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  const bool keep = fallback && a.status[k] != DPF_CASE_CONVERGED;
  if (iters) iters[k] = a.iters[k];
  if (status) status[k] = a.status[k];
  if (maxmis) maxmis[k] = keep ? a.maxmis0[k] : a.maxmis[k];
  if (loss) loss[k] = keep ? a.loss0[k] : a.loss[k];
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
int upload(T** dst, const std::vector<T>& src) {
  TRY(dalloc(dst, src.size()));
  if (!src.empty()) CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DPF_OK;
}

int num_sms_nr() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int grid_for(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)num_sms_nr() * 8)); }

}  // namespace

struct dpf_nr {
  const dpf_ybus* y = nullptr;
  int max_case = 0, Kp = 0;
  NrSymbolic sym;
  int64_t launches = 0;
  // schedule (device)
  int32_t *order = nullptr, *rank = nullptr, *frp = nullptr, *fcol = nullptr, *fdiag = nullptr,
          *ymap = nullptr, *lvl_ptr = nullptr, *rlvl_ptr = nullptr;
  int4* rows = nullptr;
  int4* targets = nullptr;
  int2* pairs = nullptr;
  // state
  double *th = nullptr, *vm = nullptr, *Ps = nullptr, *Qs = nullptr;
  double2 *V = nullptr, *U = nullptr, *I = nullptr, *X = nullptr;
  char* F = nullptr;
  char* Dinv = nullptr;
  int32_t *of = nullptr, *ot = nullptr, *active = nullptr, *status = nullptr, *iters = nullptr, *bad = nullptr,
          *n_active = nullptr;
  double2 *yff = nullptr, *yft = nullptr, *ytt = nullptr;
  double *maxmis = nullptr, *loss = nullptr, *pmax = nullptr, *psum = nullptr, *maxmis0 = nullptr,
         *loss0 = nullptr;
  int32_t* h_nact = nullptr;  // pinned
};

static void nr_release(dpf_nr* h) {
  dfree(h->order); dfree(h->rank); dfree(h->frp); dfree(h->fcol); dfree(h->fdiag);
  dfree(h->ymap); dfree(h->lvl_ptr); dfree(h->rlvl_ptr); dfree(h->rows); dfree(h->targets); dfree(h->pairs);
  dfree(h->th); dfree(h->vm); dfree(h->Ps); dfree(h->Qs); dfree(h->V); dfree(h->U); dfree(h->I); dfree(h->X);
  dfree(h->F); dfree(h->Dinv);
  dfree(h->of); dfree(h->ot); dfree(h->active); dfree(h->status); dfree(h->iters); dfree(h->bad);
  dfree(h->n_active); dfree(h->yff); dfree(h->yft); dfree(h->ytt); dfree(h->maxmis); dfree(h->loss); dfree(h->pmax); dfree(h->psum); dfree(h->maxmis0); dfree(h->loss0);
  if (h->h_nact) cudaFreeHost(h->h_nact);
  h->h_nact = nullptr;
}

static int nr_setup(dpf_nr* h) {
  const NrSymbolic& s = h->sym;
  const int n = s.n;
  const size_t npos = (size_t)s.row_ptr[n];
  TRY(upload(&h->order, s.order));
  TRY(upload(&h->rank, s.rank));
  TRY(upload(&h->frp, s.row_ptr));
  TRY(upload(&h->fcol, s.col));
  TRY(upload(&h->fdiag, s.diag));
  TRY(upload(&h->ymap, s.ymap));
  TRY(upload(&h->lvl_ptr, s.lvl_ptr));
  TRY(upload(&h->rlvl_ptr, s.rlvl_ptr));
  TRY(dalloc(&h->rows, s.rows.size() / 4));
  CK(cudaMemcpy(h->rows, s.rows.data(), s.rows.size() * 4, cudaMemcpyHostToDevice));
  TRY(dalloc(&h->targets, s.targets.size() / 4));  // two int4 per target
  CK(cudaMemcpy(h->targets, s.targets.data(), s.targets.size() * 4, cudaMemcpyHostToDevice));
  TRY(dalloc(&h->pairs, s.pairs.size() / 2));
  if (!s.pairs.empty()) CK(cudaMemcpy(h->pairs, s.pairs.data(), s.pairs.size() * 4, cudaMemcpyHostToDevice));
  const int Kp = h->Kp;
  const size_t E = (size_t)n * Kp;
  TRY(dalloc(&h->th, E)); TRY(dalloc(&h->vm, E));
  TRY(dalloc(&h->Ps, E)); TRY(dalloc(&h->Qs, E));
  TRY(dalloc(&h->V, E)); TRY(dalloc(&h->U, E)); TRY(dalloc(&h->I, E)); TRY(dalloc(&h->X, E));
  TRY(dalloc(&h->F, npos * Kp * sizeof(Blk<double>)));
  TRY(dalloc(&h->Dinv, E * sizeof(Blk<double>)));
  TRY(dalloc(&h->of, Kp)); TRY(dalloc(&h->ot, Kp)); TRY(dalloc(&h->active, Kp)); TRY(dalloc(&h->status, Kp));
  TRY(dalloc(&h->iters, Kp)); TRY(dalloc(&h->bad, Kp)); TRY(dalloc(&h->n_active, 1));
  TRY(dalloc(&h->yff, Kp)); TRY(dalloc(&h->yft, Kp)); TRY(dalloc(&h->ytt, Kp));
  TRY(dalloc(&h->maxmis, Kp)); TRY(dalloc(&h->loss, Kp));
  TRY(dalloc(&h->pmax, (size_t)NR_CHUNKS * Kp)); TRY(dalloc(&h->psum, (size_t)NR_CHUNKS * Kp));
  TRY(dalloc(&h->maxmis0, Kp)); TRY(dalloc(&h->loss0, Kp));
  CK(cudaMallocHost((void**)&h->h_nact, sizeof(int32_t)));
  return DPF_OK;
}

extern "C" int dpf_nr_create(const dpf_ybus* y, int32_t max_case, dpf_nr** out) {
  dpf::Range nvtx_range("dpf_nr_create");
  clear_error();
  if (!y || !out || max_case <= 0) return fail(DPF_E_INVALID, "dpf_nr_create: NULL argument or max_case <= 0");
  *out = nullptr;
  if (!y->dev.ready) return fail(DPF_E_STATE, "dpf_nr_create: Y_bus not uploaded (dpf_ybus_upload)");
  dpf_nr* h = new (std::nothrow) dpf_nr;
  if (!h) return fail(DPF_E_OOM, "dpf_nr_create: host allocation");
  h->y = y;
  h->max_case = max_case;
  h->Kp = (max_case + 31) / 32 * 32;
  int rc = nr_symbolic(y, (int64_t)1 << 28, &h->sym);
  if (rc == DPF_OK && (int64_t)h->sym.row_ptr[y->n] * h->Kp > ((int64_t)1 << 40) / 32)
    rc = fail(DPF_E_UNSUPPORTED, "dpf_nr_create: factor storage too large");
  if (rc == DPF_OK) rc = nr_setup(h);
  if (rc != DPF_OK) {
    nr_release(h);
    delete h;
    return rc;
  }
  *out = h;
  return DPF_OK;
}

extern "C" int dpf_nr_free(dpf_nr* h) {
  if (!h) return DPF_OK;
  nr_release(h);
  delete h;
  return DPF_OK;
}

extern "C" int dpf_nr_stats(const dpf_nr* h, int64_t* n_pos, int64_t* n_pairs, int32_t* n_levels,
                            int64_t* launches) {
  clear_error();
  if (!h) return fail(DPF_E_INVALID, "dpf_nr_stats: NULL handle");
  if (n_pos) *n_pos = h->sym.row_ptr[h->sym.n];
  if (n_pairs) *n_pairs = (int64_t)h->sym.pairs.size() / 2;
  if (n_levels) *n_levels = h->sym.n_levels;
  if (launches) *launches = h->launches;
  return DPF_OK;
}

template <class T>
static int nr_iterate_linear(dpf_nr* h, const NrArgs& a, bool smem, cudaStream_t s) {
  if (smem) {
    const size_t bytes = lu_smem_bytes<T>(a.npos, a.N);
    CK(cudaFuncSetAttribute(k_nr_lu_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k_nr_lu_smem<T><<<a.K, NR_SMEM_THREADS, bytes, s>>>(a);
    CKLAUNCH();
    h->launches += 1;
    return DPF_OK;
  }
  k_nr_assemble<T><<<grid_for((size_t)a.N * a.Kp), 256, 0, s>>>(a);
  k_nr_lu<T><<<a.Kp / a.C, NR_THREADS, 0, s>>>(a);
  CKLAUNCH();
  h->launches += 2;
  return DPF_OK;
}

static size_t smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)v;
}

extern "C" void dpf_nr_default_opts(dpf_nr_opts* o) {
  if (!o) return;
  o->precision = DPF_FP64;
  o->tol = 1e-10;
  o->max_iter = 20;
  o->flat_start = 1;
  o->lanes = 0;
  o->fallback = 0;
}

extern "C" int dpf_nr_solve(dpf_nr* h, const dpf_batch* b, const dpf_nr_opts* o, void* stream) {
  dpf::Range nvtx_range("dpf_nr_solve");
  clear_error();
  if (!h || !b || !o) return fail(DPF_E_INVALID, "dpf_nr_solve: NULL argument");
  const int precision = o->precision, max_iter = o->max_iter, flat_start = o->flat_start;
  const double tol = o->tol;
  if (o->lanes < 0 || o->lanes > 32 || (o->lanes & (o->lanes - 1)))
    return fail(DPF_E_INVALID, "dpf_nr_solve: lanes must be 0 or a power of 2 up to 32");
  const dpf_ybus* y = h->y;
  const int K = b->n_case;
  if (K <= 0 || K > h->max_case) return fail(DPF_E_INVALID, "dpf_nr_solve: n_case %d outside 1..%d", K, h->max_case);
  if (b->host_io) return fail(DPF_E_INVALID, "dpf_nr_solve: device pointers only (host_io = 0)");
  if (!b->va || !b->vm) return fail(DPF_E_INVALID, "dpf_nr_solve: va and vm are required");
  if (b->va_start || b->vm_start) return fail(DPF_E_INVALID, "dpf_nr_solve: va_start / vm_start are not supported");
  if ((b->p_spec == nullptr) != (b->q_spec == nullptr))
    return fail(DPF_E_INVALID, "dpf_nr_solve: p_spec and q_spec are given together");
  if (precision != DPF_FP32 && precision != DPF_FP64)
    return fail(DPF_E_INVALID, "dpf_nr_solve: precision must be DPF_FP32 or DPF_FP64");
  if (!(tol >= 0.0) || max_iter < 0) return fail(DPF_E_INVALID, "dpf_nr_solve: tol >= 0 and max_iter >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->outage) {
    std::vector<int32_t> ho(K);
    CK(cudaMemcpyAsync(ho.data(), b->outage, (size_t)K * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < K; ++k) {
      const int l = ho[k];
      if (l < -1 || l >= y->m) return fail(DPF_E_INVALID, "case %d: outage index %d out of range", k, l);
      if (l >= 0 && y->bridge[l]) return fail(DPF_E_ISLANDED, "case %d: removing branch %d islands the grid", k, l);
    }
  }
  const DeviceYbus& d = y->dev;
  const NrSymbolic& sym = h->sym;
  NrArgs a;
  memset(&a, 0, sizeof a);
  a.N = y->n;
  a.K = K;
  a.Kp = (K + 31) / 32 * 32;
  // cases per CTA: the C lanes of a slot share its schedule loads and read
  // C consecutive blocks; few enough cases per CTA that every CTA of the
  // batch is resident at once (each walks the whole tree: a second wave
  // would double the time)
  const int C_fixed = o->lanes;
  auto lanes_for = [&](int n_active) {
    if (C_fixed) return C_fixed;
    int C = 4;
    while (C > 1 && n_active / C < num_sms_nr()) C >>= 1;
    return C;
  };
  a.C = lanes_for(K);
  // The shared-memory form where one case's factor fits and the cases still
  // iterating fit in one wave of one CTA per SM (its walk down the tree is
  // shorter, but a second wave would double it); else the global-memory
  // form.  Both give the same bits.  o->lanes > 0 forces the global form.
  const size_t need = precision == DPF_FP64 ? lu_smem_bytes<double>(sym.row_ptr[sym.n], y->n)
                                            : lu_smem_bytes<float>(sym.row_ptr[sym.n], y->n);
  const bool fits = o->lanes == 0 && need <= smem_optin();
  bool smem = false;
  a.va_slack = y->va_slack;
  a.tol = tol;
  a.inv_m = y->m_loss > 0 ? 1.0 / y->m_loss : 0.0;
  a.max_iter = max_iter;
  a.rp = d.row_ptr;
  a.ycol = d.col;
  a.yval = d.val64;
  a.type = d.type;
  a.p64 = d.p64;
  a.q64 = d.q64;
  a.vmset = d.vmset;
  a.perm = d.perm;
  a.order = h->order;
  a.rank = h->rank;
  a.frp = h->frp;
  a.fcol = h->fcol;
  a.fdiag = h->fdiag;
  a.ymap = h->ymap;
  a.n_levels = sym.n_levels;
  a.lvl_ptr = h->lvl_ptr;
  a.targets = h->targets;
  a.pairs = h->pairs;
  a.rlvl_ptr = h->rlvl_ptr;
  a.rows = h->rows;
  a.npos = sym.row_ptr[sym.n];
  a.th = h->th;
  a.vm = h->vm;
  a.V = h->V;
  a.U = h->U;
  a.I = h->I;
  a.X = h->X;
  a.Ps = b->p_spec ? h->Ps : nullptr;
  a.Qs = b->p_spec ? h->Qs : nullptr;
  a.F = h->F;
  a.Dinv = h->Dinv;
  a.of = h->of;
  a.ot = h->ot;
  a.yff = h->yff;
  a.yft = h->yft;
  a.ytt = h->ytt;
  a.active = h->active;
  a.status = h->status;
  a.iters = h->iters;
  a.bad = h->bad;
  a.maxmis = h->maxmis;
  a.loss = h->loss;
  a.n_active = h->n_active;
  a.pmax = h->pmax;
  a.psum = h->psum;
  a.maxmis0 = h->maxmis0;
  a.loss0 = h->loss0;
  const size_t E = (size_t)a.N * a.Kp;
  const int cb = (a.Kp + 255) / 256;
  k_nr_init<<<cb, 256, 0, s>>>(a, b->outage, d.br_f, d.br_t, d.br_r, d.br_x, d.br_bch, d.br_tap);
  k_nr_in<<<grid_for(E), 256, 0, s>>>(a, b->va, b->vm, b->p_spec, b->q_spec, b->vm_set, flat_start ? 1 : 0);
  CKLAUNCH();
  h->launches += 2;
  for (int it = 0;; ++it) {
    k_nr_volt<<<grid_for(E), 256, 0, s>>>(a);
    k_nr_eval<<<grid_for(E), 256, 0, s>>>(a);
    CK(cudaMemsetAsync(a.n_active, 0, 4, s));
    k_nr_partial<<<dim3(a.Kp / 32, NR_CHUNKS), 256, 0, s>>>(a);
    a.first = it == 0;
    k_nr_check<<<cb, 256, 0, s>>>(a);
    CKLAUNCH();
    h->launches += 4;
    CK(cudaMemcpyAsync(h->h_nact, a.n_active, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*h->h_nact == 0 || it > max_iter) break;
    // few cases left: fewer cases per CTA, more slots per case (a shorter
    // walk for each; CTAs whose cases have all stopped return at once)
    a.C = lanes_for(*h->h_nact);
    smem = fits && *h->h_nact <= num_sms_nr();
    if (precision == DPF_FP64) TRY(nr_iterate_linear<double>(h, a, smem, s));
    else TRY(nr_iterate_linear<float>(h, a, smem, s));
    k_nr_update<<<grid_for(E), 256, 0, s>>>(a);
    CKLAUNCH();
    h->launches += 1;
  }
  const int fb = o->fallback && !flat_start;
  k_nr_out<<<grid_for(E), 256, 0, s>>>(a, b->va, b->vm, fb);
  k_nr_case_out<<<cb, 256, 0, s>>>(a, b->iters, b->status, b->max_mismatch, b->loss, fb);
  CKLAUNCH();
  h->launches += 2;
  return DPF_OK;
}
