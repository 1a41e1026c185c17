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
// Solver: conjugate gradients with the Jacobi preconditioner, all cases at
// once in the case-minor layout (element (i, k) at i*Kp + k), each CTA on a
// contiguous block of rows.  One iteration is two launches:
//   k_dc_spmv_dir     the new direction p' = z + beta p and q' = B' p', formed
//                     as B' z + beta q from the previous q = B' p (so no CTA
//                     waits for another's p' and p is never gathered), and the
//                     per-case partial sums of p'.q'
//   k_dc_update_case  alpha = rz / pq; x += alpha p'; r -= alpha q';
//                     z = r / diag(B'); partial sums of r.z and r.r; the last
//                     CTA of each case tile then takes the per-case step:
//                     stop when |r| <= tol |r0|, else beta = rz' / rz
// The recurrence for q' is the same arithmetic as B' p' up to rounding.  The
// two direction buffers alternate.  Slack rows are not unknowns: their r, z,
// p stay 0 and their x holds the slack angle.
//
// Outage shift (dc_start with a warm start): the right-hand side of case k is
// the outaged branch's DC flow at the case's start angles, c_k = b_l
// (theta_f - theta_t), put back at its ends (+c_k at f, -c_k at t, 0 elsewhere)
// and x0 = 0 everywhere, so x is the angle change B'^-1 (B - B') theta that
// removing the branch causes in the DC model; it is added to the start angles.
//
// Precision.  GB300 issues FP64 at a small fraction of its FP32 rate, and in
// FP64 this loop kept the FP64 pipe 73-86% busy.  So the vectors are double-float:
// an unevaluated sum hi + lo of two floats (about 48 significant bits, far
// below the 1e-10 residual the solver is asked for), in the same 8 bytes as a
// double, with per-element arithmetic built from the error-free
// transformations of Knuth (two-sum) and Dekker (two-product, here with an
// FMA), as in the double-double arithmetic of Hida, Li and Bailey.  B and
// 1 / B_ii are uploaded as hi/lo pairs; the per-case scalars (alpha, beta, the
// dot products' totals, the stop test) stay FP64.  x is widened to FP64 at the
// end.  A solve asked for a relative residual of 1e-5 or more (a start for
// the DPF iterations, not an answer) runs the same kernels on plain FP32
// vectors (T = float: half the bytes, no two-sums), B and 1 / B_ii their
// high words.
#pragma once

#include "dpf_kernels.cuh"

namespace dpf {

// ---- double-float arithmetic (float2: x = hi, y = lo, |lo| <= ulp(hi) / 2) --
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 df_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// a + b with one two-sum of the high words and the low words added plainly:
// its error is about 2^-48 of |a| + |b| (not of the result), ample for a
// residual asked to fall to 1e-10 of the initial one
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 s = df_two_sum(a.x, b.x);
  return df_quick(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return df_quick(p, e);
}
__device__ __forceinline__ float2 df_fma(float2 a, float2 b, float2 c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_from(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
// a / b: the quotient of the high words refined by one correction step
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
  const float q0 = __fdiv_rn(a.x, b.x);
  const float2 r = df_add(a, df_neg(df_mul(make_float2(q0, 0.f), b)));
  return df_quick(q0, __fdiv_rn(r.x, b.x));
}
// The same operations on plain FP32 vectors (T = float).
__device__ __forceinline__ float df_add(float a, float b) { return a + b; }
__device__ __forceinline__ float df_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float df_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float df_neg(float a) { return -a; }
__device__ __forceinline__ double df_val(float a) { return (double)a; }
__device__ __forceinline__ float df_div(float a, float b) { return __fdiv_rn(a, b); }
template <class T> __device__ __forceinline__ T df_cast(double v);
template <> __device__ __forceinline__ float2 df_cast<float2>(double v) { return df_from(v); }
template <> __device__ __forceinline__ float df_cast<float>(double v) { return (float)v; }
// B entries (uploaded as hi/lo pairs) in the vector type
template <class T> __device__ __forceinline__ T df_coef(float2 v);
template <> __device__ __forceinline__ float2 df_coef<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ float df_coef<float>(float2 v) { return v.x; }
template <class T> __device__ __forceinline__ T df_zero();
template <> __device__ __forceinline__ float2 df_zero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ float df_zero<float>() { return 0.f; }

// rows per thread and step of the two iteration kernels on FP32 vectors
// (double-float vectors take one: four cost them occupancy, 125 -> 134 us)
#ifndef DC_ROWS_F32
#define DC_ROWS_F32 4
#endif
template <class T> struct DCRows { static constexpr int n = sizeof(T) == 4 ? DC_ROWS_F32 : 1; };

template <class T> struct DCArgs {
  int N, Kp, lanes, K;
  const int32_t* __restrict__ rp;
  const int32_t* __restrict__ col;
  const float2* __restrict__ bval;   // B values in CSR order (hi, lo)
  const int32_t* __restrict__ dpos;  // position of each row's diagonal entry
  const float2* __restrict__ dinv;   // [N] 1 / B_ii (hi, lo)
  const uint8_t* __restrict__ type;
  const double* pspec;  // [N][Kp] per case or [N]
  int spec_per_case;
  double va_slack;
  const int32_t* of;  // per case: internal from/to bus of the outaged branch (-1: none)
  const int32_t* ot;
  double* ob;         // per case: its susceptance b_l
  const double* flow; // per case: c_k of the outage shift (NULL: solve B' x = P)
  T* x;            // vectors [N][Kp] (double-float pairs or FP32)
  T* r;
  T* z;
  T* p;            // direction of the previous iteration
  T* p_new;        // direction of this iteration
  T* q;            // B' p of the previous iteration, then of this one
  int rpb;                  // rows per CTA
  unsigned int* tile_cnt;   // per case tile: CTAs done with the update (reset by the last)
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

// (B' v)_i for case k (v in the case-minor layout); ob2 = the outaged
// branch's b_l in the vector type.
template <class T>
__device__ __forceinline__ T dc_row(const DCArgs<T>& a, const T* __restrict__ v, int i, int k, size_t Kp, int of,
                                    int ot, T ob2) {
  T s = df_zero<T>();
  const int p1 = __ldg(a.rp + i + 1);
  for (int p = __ldg(a.rp + i); p < p1; ++p)
    s = df_fma(df_coef<T>(__ldg(a.bval + p)), v[(size_t)__ldg(a.col + p) * Kp + k], s);
  if (i == of || i == ot) {
    const T d = df_add(v[(size_t)of * Kp + k], df_neg(v[(size_t)ot * Kp + k]));  // v_f - v_t
    s = df_fma(i == of ? df_neg(ob2) : ob2, d, s);
  }
  return s;
}

// Jacobi step z_i = r_i / B'_ii.
template <class T>
__device__ __forceinline__ T dc_jacobi(const DCArgs<T>& a, T r, int i, int of, int ot, T ob2) {
  if (i == of || i == ot) return df_div(r, df_add(df_coef<T>(__ldg(a.bval + __ldg(a.dpos + i))), df_neg(ob2)));
  return df_mul(r, df_coef<T>(__ldg(a.dinv + i)));
}

// Per case: the outaged branch's susceptance, the solver state reset.
template <class T>
__global__ void k_dc_case_init(DCArgs<T> a, const int32_t* __restrict__ outage, const double* __restrict__ br_x,
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

// x0 (slack angle at slack buses, 0 elsewhere) for every element; p, q zeroed.
template <class T>
__global__ void k_dc_x0(DCArgs<T> a) {
  const size_t n = (size_t)a.N * a.Kp;
  const T zero = df_zero<T>(), vs = df_cast<T>(a.va_slack);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.Kp);
    a.x[e] = (__ldg(a.type + i) == BUS_SLACK) ? vs : zero;
    a.p[e] = zero;
    a.p_new[e] = zero;
    a.q[e] = zero;  // q' = B' z + beta q reads it with beta = 0 first
  }
}

// r0 = P - B' x0 at the unknowns, z0 = r0 / diag, p0 = z0; sums r.z, r.r.
template <class T>
__global__ void __launch_bounds__(1024) k_dc_start(DCArgs<T> a) {
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  const size_t Kp = (size_t)a.Kp;
  T rz = df_zero<T>(), rr = rz;
  if (k < a.Kp && a.active[k]) {
    const int of = a.of ? a.of[k] : -1, ot = a.ot ? a.ot[k] : -1;
    const T ob2 = df_cast<T>(a.ob[k]);
    for (int i = mp.row0; i < a.N; i += mp.rstride) {
      const size_t e = (size_t)i * Kp + k;
      T r = df_zero<T>(), z = r;
      if (__ldg(a.type + i) != BUS_SLACK) {
        const double Pi = a.flow ? (i == of ? a.flow[k] : i == ot ? -a.flow[k] : 0.0)
                                 : (a.spec_per_case ? a.pspec[e] : a.pspec[i]);
        const T P = df_cast<T>(Pi);
        r = df_add(P, df_neg(dc_row(a, a.x, i, k, Kp, of, ot, ob2)));
        z = dc_jacobi(a, r, i, of, ot, ob2);
      }
      a.r[e] = r;
      a.z[e] = z;
      a.p[e] = z;
      rz = df_fma(r, z, rz);
      rr = df_fma(r, r, rr);
    }
  }
  case_sum2_atomic(df_val(rz), df_val(rr), a.lanes, a.rz, a.rr0, a.Kp);
}

template <class T>
__global__ void __launch_bounds__(256) k_dc_spmv_dir(DCArgs<T> a) {
  const BMap mp = block_map(a.lanes, a.N, a.rpb);
  const int k = mp.k;
  const size_t Kp = (size_t)a.Kp;
  T pq = df_zero<T>();
  if (k < a.Kp && a.active[k]) {
    const int of = a.of ? a.of[k] : -1, ot = a.ot ? a.ot[k] : -1;
    const T ob2 = df_cast<T>(a.ob[k]), beta = df_cast<T>(a.beta[k]);
    // DCRows rows per step: their loads and gathers are issued before any
    // result is stored (more requests in flight per thread)
    for (int i0 = mp.i0; i0 < mp.r1; i0 += DCRows<T>::n * mp.istride) {
      T pv[DCRows<T>::n], zv[DCRows<T>::n], qv[DCRows<T>::n], bz[DCRows<T>::n];
      bool on[DCRows<T>::n];
#pragma unroll
      for (int u = 0; u < DCRows<T>::n; ++u) {
        const int i = i0 + u * mp.istride;
        on[u] = i < mp.r1 && __ldg(a.type + i) != BUS_SLACK;  // p, q stay 0 at slack rows
        if (on[u]) {
          const size_t e = (size_t)i * Kp + k;
          pv[u] = a.p[e];
          zv[u] = a.z[e];
          qv[u] = a.q[e];
        }
      }
#pragma unroll
      for (int u = 0; u < DCRows<T>::n; ++u)
        if (on[u]) bz[u] = dc_row(a, a.z, i0 + u * mp.istride, k, Kp, of, ot, ob2);
#pragma unroll
      for (int u = 0; u < DCRows<T>::n; ++u) {
        if (!on[u]) continue;
        const size_t e = (size_t)(i0 + u * mp.istride) * Kp + k;
        const T pn = df_fma(beta, pv[u], zv[u]);
        const T q = df_fma(beta, qv[u], bz[u]);
        a.p_new[e] = pn;
        a.q[e] = q;
        pq = df_fma(pn, q, pq);
      }
    }
  }
  case_sum2_atomic(df_val(pq), 0.0, a.lanes, a.pq, nullptr, a.Kp);
}

// Per case, after all row blocks' sums: convergence test and the next beta.
template <class T>
__device__ __forceinline__ void dc_case_step(const DCArgs<T>& a, int k) {
  if (a.active[k]) {
    a.iters[k] += 1;
    const double rr = __ldcg(a.rr + k), rr0 = __ldcg(a.rr0 + k), rzn = __ldcg(a.rzn + k);
    a.res[k] = rr0 > 0.0 ? sqrt(rr / rr0) : 0.0;
    if (rr <= a.tol2 * rr0 || !(rr == rr)) {  // converged (or broken down: NaN)
      a.active[k] = 0;
      atomicSub(a.n_active, 1);
    } else {
      const double rz = __ldcg(a.rz + k);
      a.beta[k] = rz != 0.0 ? rzn / rz : 0.0;
      a.rz[k] = rzn;
    }
  }
  a.rzn[k] = 0.0;
  a.pq[k] = 0.0;
  a.rr[k] = 0.0;
}

template <class T>
__global__ void __launch_bounds__(256) k_dc_update_case(DCArgs<T> a) {
  const BMap mp = block_map(a.lanes, a.N, a.rpb);
  const int k = mp.k;
  const size_t Kp = (size_t)a.Kp;
  // alpha = rz / pq once per case of the tile (an FP64 divide is dear here),
  // shared with the CTA's other threads of that case
  __shared__ double s_alpha[32];
  if ((int)threadIdx.x < a.lanes) {
    const int kk = blockIdx.x * a.lanes + threadIdx.x;
    double al = 0.0;
    if (kk < a.Kp) {
      const double pq = __ldcg(a.pq + kk);
      al = pq != 0.0 ? __ldcg(a.rz + kk) / pq : 0.0;
    }
    s_alpha[threadIdx.x] = al;
  }
  __syncthreads();
  T rz = df_zero<T>(), rr = rz;
  if (k < a.Kp && a.active[k]) {
    const int of = a.of ? a.of[k] : -1, ot = a.ot ? a.ot[k] : -1;
    const T ob2 = df_cast<T>(a.ob[k]);
    const T alpha = df_cast<T>(s_alpha[mp.kl]), nalpha = df_neg(alpha);
    for (int i0 = mp.i0; i0 < mp.r1; i0 += DCRows<T>::n * mp.istride) {
      T pv[DCRows<T>::n], qv[DCRows<T>::n], xv[DCRows<T>::n], rv[DCRows<T>::n];
      bool on[DCRows<T>::n];
#pragma unroll
      for (int u = 0; u < DCRows<T>::n; ++u) {
        const int i = i0 + u * mp.istride;
        on[u] = i < mp.r1 && __ldg(a.type + i) != BUS_SLACK;
        if (on[u]) {
          const size_t e = (size_t)i * Kp + k;
          pv[u] = a.p_new[e];
          qv[u] = a.q[e];
          xv[u] = a.x[e];
          rv[u] = a.r[e];
        }
      }
#pragma unroll
      for (int u = 0; u < DCRows<T>::n; ++u) {
        if (!on[u]) continue;
        const int i = i0 + u * mp.istride;
        const size_t e = (size_t)i * Kp + k;
        a.x[e] = df_fma(alpha, pv[u], xv[u]);
        const T r = df_fma(nalpha, qv[u], rv[u]);
        const T z = dc_jacobi(a, r, i, of, ot, ob2);
        a.r[e] = r;
        a.z[e] = z;
        rz = df_fma(r, z, rz);
        rr = df_fma(r, r, rr);
      }
    }
  }
  case_sum2_atomic(df_val(rz), df_val(rr), a.lanes, a.rzn, a.rr, a.Kp);
  // the last CTA of the case tile (every CTA counts itself after fencing its
  // atomics) takes the per-case step for the tile's cases
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(a.tile_cnt + blockIdx.x, 1u);
    last = (prev == gridDim.y - 1);
    if (last) a.tile_cnt[blockIdx.x] = 0u;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int c = threadIdx.x; c < a.lanes; c += blockDim.x) {
      const int kk = blockIdx.x * a.lanes + c;
      if (kk < a.Kp) dc_case_step(a, kk);
    }
  }
}

// The solution widened to FP64: in place for double-float pairs (each
// element's 8 bytes are read before they are written), into `out` for FP32.
template <class T>
__global__ void k_dc_widen(T* x, double* out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const T v = x[e];
    out[e] = df_val(v);
  }
}

// Outage shift: c_k = b_l (theta_f - theta_t) from case k's start angles in
// the master state (0 for a case without an outage).  After k_dc_case_init.
template <class R>
__global__ void k_dc_flow(const typename Prec<R>::MS* __restrict__ ms, const int32_t* __restrict__ of,
                          const int32_t* __restrict__ ot, const double* __restrict__ ob, double* __restrict__ flow,
                          int K, int Kp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Kp) return;
  const int f = k < K ? of[k] : -1, t = k < K ? ot[k] : -1;
  flow[k] = (f >= 0 && t >= 0)
                ? ob[k] * (mval(ms_th(ms[(size_t)f * Kp + k])) - mval(ms_th(ms[(size_t)t * Kp + k])))
                : 0.0;
}

// DPF started from the DC angles: theta = x (add = 0) or theta + x (add = 1,
// the outage shift) at the pv and pq buses, |V| as initialised, V rebuilt
// from the master pair.
template <class R>
__global__ void k_dc_apply(const double* __restrict__ x, typename Prec<R>::MS* __restrict__ ms,
                           typename Prec<R>::C* __restrict__ V, const uint8_t* __restrict__ type, int N, int K,
                           int Kp, int add) {
  using M = typename Prec<R>::M;
  const size_t n = (size_t)N * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Kp), k = (int)(e % Kp);
    if (k >= K || __ldg(type + i) == BUS_SLACK) continue;
    const M th = mfrom<M>(add ? mval(ms_th(ms[e])) + x[e] : x[e]);
    const M vm = ms_vm(ms[e]);
    ms[e] = ms_make(th, vm);
    V[e] = volt(th, vm);
  }
}

}  // namespace dpf
