// DC approximation of the power flow on the GPU: B theta = P for many cases.
//
// The comparison model and optional initialisation of Sec. 2 / Alg. 2: with
// |V| = 1, no resistance, no charging and small angle differences, branch
// l = (f, t) carries b_l (theta_f - theta_t) with b_l = 1 / (x_l tau_l), so
// the angles of the pv and pq buses solve B theta = P (slack angles fixed, one
// slack per island).  B has the sparsity of Y_bus; its values are uploaded with
// Y_bus.  An outaged branch is the rank-one correction
// B' = B - b_l (e_f - e_t)(e_f - e_t)^T of the shared B, as for the N-1 Y_bus.
//
// Solver: conjugate gradients with the Jacobi preconditioner, in FP64, all
// cases at once in the case-minor layout (element (i, k) at i*Kp + k).  One
// iteration is four launches:
//   k_dc_spmv    q = B' p and the per-case partial sums of p.q
//   k_dc_update  alpha = rz / pq; x += alpha p; r -= alpha q; z = r / diag(B');
//                partial sums of r.z and r.r
//   k_dc_case    per case: stop when |r| <= tol |r0|, else beta = rz' / rz
//   k_dc_dir     p = z + beta p
// Slack rows are not unknowns: their r, z, p stay 0 and their x holds the
// slack angle.
#pragma once

#include "dpf_kernels.cuh"

namespace dpf {

struct DCArgs {
  int N, Kp, lanes, K;
  const int32_t* __restrict__ rp;
  const int32_t* __restrict__ col;
  const double* __restrict__ bval;  // B values in CSR order
  const int32_t* __restrict__ dpos;  // position of each row's diagonal entry
  const uint8_t* __restrict__ type;
  const double* pspec;  // [N][Kp] per case or [N]
  int spec_per_case;
  double va_slack;
  const int32_t* of;  // per case: internal from/to bus of the outaged branch (-1: none)
  const int32_t* ot;
  double* ob;         // per case: its susceptance b_l
  double* x;
  double* r;
  double* z;
  double* p;
  double* q;
  // per case
  double* rz;
  double* rzn;
  double* pq;
  double* rr;
  double* rr0;
  double* beta;
  double* res;   // final |r| / |r0|
  int32_t* active;
  int32_t* iters;
  int32_t* n_active;
  double tol2;  // tol^2
};

// Per-case sums of two values over the CTA's threads, one atomic each per case.
__device__ __forceinline__ void case_sum2_atomic(double a, double b, int lanes, double* oa, double* ob, int Kp) {
  __shared__ double ra[32][32];
  __shared__ double rb[32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int off = 16; off >= lanes; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if (lane < lanes) {
    ra[warp][lane] = a;
    rb[warp][lane] = b;
  }
  __syncthreads();
  if (threadIdx.x < lanes) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < wpb; ++w) {
      sa += ra[w][threadIdx.x];
      sb += rb[w][threadIdx.x];
    }
    const int k = blockIdx.x * lanes + threadIdx.x;
    if (k < Kp) {
      if (oa && sa != 0.0) atomicAdd(oa + k, sa);
      if (ob && sb != 0.0) atomicAdd(ob + k, sb);
    }
  }
}

// (B' v)_i for case k (v in the case-minor layout).
__device__ __forceinline__ double dc_row(const DCArgs& a, const double* __restrict__ v, int i, int k, size_t Kp,
                                         int of, int ot, double ob) {
  double s = 0.0;
  const int p1 = __ldg(a.rp + i + 1);
  for (int p = __ldg(a.rp + i); p < p1; ++p) s = fma(__ldg(a.bval + p), v[(size_t)__ldg(a.col + p) * Kp + k], s);
  if (i == of) s -= ob * (v[(size_t)of * Kp + k] - v[(size_t)ot * Kp + k]);
  else if (i == ot) s -= ob * (v[(size_t)ot * Kp + k] - v[(size_t)of * Kp + k]);
  return s;
}

__device__ __forceinline__ double dc_diag(const DCArgs& a, int i, int of, int ot, double ob) {
  const double d = __ldg(a.bval + __ldg(a.dpos + i));
  return (i == of || i == ot) ? d - ob : d;
}

// Per case: the outaged branch's susceptance, the solver state reset.
__global__ void k_dc_case_init(DCArgs a, const int32_t* __restrict__ outage, const double* __restrict__ br_x,
                               const double* __restrict__ br_tap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.Kp) return;
  const int ell = (k < a.K && outage) ? outage[k] : -1;
  a.ob[k] = ell >= 0 ? 1.0 / (br_x[ell] * (br_tap[ell] == 0.0 ? 1.0 : br_tap[ell])) : 0.0;
  a.active[k] = k < a.K ? 1 : 0;
  a.iters[k] = 0;
  a.rz[k] = a.rzn[k] = a.pq[k] = a.rr[k] = a.rr0[k] = 0.0;
  a.beta[k] = 0.0;
  a.res[k] = 0.0;
}

// x0 (slack angle at slack buses, 0 elsewhere) for every element.
__global__ void k_dc_x0(DCArgs a) {
  const size_t n = (size_t)a.N * a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.Kp);
    a.x[e] = (__ldg(a.type + i) == BUS_SLACK) ? a.va_slack : 0.0;
    a.p[e] = 0.0;
  }
}

// r0 = P - B' x0 at the unknowns, z0 = r0 / diag, p0 = z0; sums r.z, r.r.
__global__ void __launch_bounds__(1024) k_dc_start(DCArgs a) {
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  const size_t Kp = (size_t)a.Kp;
  double rz = 0.0, rr = 0.0;
  if (k < a.Kp && a.active[k]) {
    const int of = a.of ? a.of[k] : -1, ot = a.ot ? a.ot[k] : -1;
    const double ob = a.ob[k];
    for (int i = mp.row0; i < a.N; i += mp.rstride) {
      const size_t e = (size_t)i * Kp + k;
      double r = 0.0, z = 0.0;
      if (__ldg(a.type + i) != BUS_SLACK) {
        const double P = a.spec_per_case ? a.pspec[e] : a.pspec[i];
        r = P - dc_row(a, a.x, i, k, Kp, of, ot, ob);
        z = r / dc_diag(a, i, of, ot, ob);
      }
      a.r[e] = r;
      a.z[e] = z;
      a.p[e] = z;
      rz = fma(r, z, rz);
      rr = fma(r, r, rr);
    }
  }
  case_sum2_atomic(rz, rr, a.lanes, a.rz, a.rr0, a.Kp);
}

__global__ void __launch_bounds__(1024) k_dc_spmv(DCArgs a) {
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  const size_t Kp = (size_t)a.Kp;
  double pq = 0.0;
  if (k < a.Kp && a.active[k]) {
    const int of = a.of ? a.of[k] : -1, ot = a.ot ? a.ot[k] : -1;
    const double ob = a.ob[k];
    for (int i = mp.row0; i < a.N; i += mp.rstride) {
      const size_t e = (size_t)i * Kp + k;
      const double q = (__ldg(a.type + i) != BUS_SLACK) ? dc_row(a, a.p, i, k, Kp, of, ot, ob) : 0.0;
      a.q[e] = q;
      pq = fma(a.p[e], q, pq);
    }
  }
  case_sum2_atomic(pq, 0.0, a.lanes, a.pq, nullptr, a.Kp);
}

__global__ void __launch_bounds__(1024) k_dc_update(DCArgs a) {
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  const size_t Kp = (size_t)a.Kp;
  double rz = 0.0, rr = 0.0;
  if (k < a.Kp && a.active[k]) {
    const int of = a.of ? a.of[k] : -1, ot = a.ot ? a.ot[k] : -1;
    const double ob = a.ob[k];
    const double alpha = a.pq[k] != 0.0 ? a.rz[k] / a.pq[k] : 0.0;
    for (int i = mp.row0; i < a.N; i += mp.rstride) {
      if (__ldg(a.type + i) == BUS_SLACK) continue;
      const size_t e = (size_t)i * Kp + k;
      a.x[e] = fma(alpha, a.p[e], a.x[e]);
      const double r = fma(-alpha, a.q[e], a.r[e]);
      const double z = r / dc_diag(a, i, of, ot, ob);
      a.r[e] = r;
      a.z[e] = z;
      rz = fma(r, z, rz);
      rr = fma(r, r, rr);
    }
  }
  case_sum2_atomic(rz, rr, a.lanes, a.rzn, a.rr, a.Kp);
}

// One thread per case: convergence test and the next direction's beta.
__global__ void k_dc_case(DCArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.Kp) return;
  if (a.active[k]) {
    a.iters[k] += 1;
    const double rr = a.rr[k], rr0 = a.rr0[k];
    a.res[k] = rr0 > 0.0 ? sqrt(rr / rr0) : 0.0;
    if (rr <= a.tol2 * rr0 || !(rr == rr)) {  // converged (or broken down: NaN)
      a.active[k] = 0;
      atomicSub(a.n_active, 1);
    } else {
      a.beta[k] = a.rz[k] != 0.0 ? a.rzn[k] / a.rz[k] : 0.0;
      a.rz[k] = a.rzn[k];
    }
  }
  a.rzn[k] = 0.0;
  a.pq[k] = 0.0;
  a.rr[k] = 0.0;
}

__global__ void __launch_bounds__(1024) k_dc_dir(DCArgs a) {
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  if (k >= a.Kp || !a.active[k]) return;
  const size_t Kp = (size_t)a.Kp;
  const double beta = a.beta[k];
  for (int i = mp.row0; i < a.N; i += mp.rstride) {
    const size_t e = (size_t)i * Kp + k;
    a.p[e] = fma(beta, a.p[e], a.z[e]);
  }
}

// DPF started from the DC angles: theta = x at the pv and pq buses (|V| as
// initialised), V rebuilt from the master pair.
template <class R>
__global__ void k_dc_apply(const double* __restrict__ x, typename Prec<R>::MS* __restrict__ ms,
                           typename Prec<R>::C* __restrict__ V, const uint8_t* __restrict__ type, int N, int K,
                           int Kp) {
  using M = typename Prec<R>::M;
  const size_t n = (size_t)N * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Kp), k = (int)(e % Kp);
    if (k >= K || __ldg(type + i) == BUS_SLACK) continue;
    const M th = mfrom<M>(x[e]);
    const M vm = ms_vm(ms[e]);
    ms[e] = ms_make(th, vm);
    V[e] = volt(th, vm);
  }
}

}  // namespace dpf
