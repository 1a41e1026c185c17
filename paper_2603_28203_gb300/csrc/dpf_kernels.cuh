// Device kernels of the DPF hot path (sm_103a).
//
// Layout: per-case state is stored case-minor, element (bus i, case k) at
// i*Kp + k, with Kp the case count padded to the lane group.  A warp covers
// `lanes` consecutive cases of 32/lanes consecutive buses, so for a batch of
// >= 32 cases all 32 lanes work on one bus: the Y_bus row is read once per
// warp (a broadcast 16-byte load per nonzero) and every gather of a
// neighbour's voltage is one coalesced 256-byte (FP32) access.  For a single
// case (lanes = 1) the same code is a thread-per-row CSR SpMV.
//
// One DPF iteration (Alg. 1) is two launches:
//   k_fwd   I = Y V (+ N-1 correction), S = V conj(I), dP/dQ, loss partials,
//           w = c conj(V); the last CTA of each case tile then runs the
//           per-case scheduler (loss, ReduceLROnPlateau / StepLR, the step's
//           bias-corrected terms)            (Eq. powerbalance, Alg. 1)
//   k_adj   z = Y w (+ N-1 correction), h = conj(c) S + V z (conj(c) S
//           rebuilt from w), dL/dtheta = -Im h, dL/d|V| = Re h / |V|,
//           optimiser update, new V
// and every `check_every` iterations the FP64 test k_volt64 + k_check64 +
// k_apply (max |f| per case <= tol -> the case stops).
//
// The adjoint identity used by k_adj: with c_i = (2/m)(dP_i + j dQ_i),
// dL = Re sum_i conj(c_i) dS_i and dS_i = dV_i conj(I_i) + V_i conj((Y dV)_i),
// so dL = Re sum_k dV_k (conj(c_k I_k) + (Y^T w)_k) with w = c conj(V).  Y is
// symmetric (no phase shifters), and dV_k = V_k (j dtheta_k + d|V_k|/|V_k|).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dpf {

enum { BUS_PQ = 0, BUS_PV = 1, BUS_SLACK = 2 };
enum { CASE_CONVERGED = 0, CASE_MAX_ITER = 1, CASE_DIVERGED = 2 };
enum { SCHED_CONST = 0, SCHED_PLATEAU = 1, SCHED_STEP = 2 };
enum { OPT_ADAM = 0, OPT_SGD = 1, OPT_RMSPROP = 2 };

template <class R> struct Prec;
// C: complex working value; M: master value (FP32 mode: (hi, lo) double-float);
// MS: one element's master pair (theta, |V|) in one 16-byte word
template <> struct Prec<float> { using C = float2; using M = float2; using MS = float4; };
template <> struct Prec<double> { using C = double2; using M = double; using MS = double2; };

// One element's optimiser moments: (m, v) of theta, then of |V| (pq buses).
// Stored interleaved so that an element's state is one aligned access.
template <class R> struct __align__(4 * sizeof(R) >= 16 ? 16 : 4 * sizeof(R)) Mom { R m1, v1, m2, v2; };

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float sqrtT(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrtT(double a) { return sqrt(a); }
// Optimiser arithmetic: in FP32 an approximate sqrt (rsqrt, ~1 ulp) and a
// fast division (~2 ulp); the result only scales an optimiser step.  FP64
// keeps IEEE operations.
__device__ __forceinline__ float sqrt_step(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }
__device__ __forceinline__ double sqrt_step(double v) { return sqrt(v); }
__device__ __forceinline__ float div_step(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_step(double a, double b) { return a / b; }
// a*b + c in an optimiser's moment update: fused in FP32; in FP64 a rounded
// product and a rounded sum, as the textbook update the FP64 path is checked
// against writes it.
__device__ __forceinline__ float madd_step(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd_step(double a, double b, double c) { return __dadd_rn(__dmul_rn(a, b), c); }

// acc += y * v (complex)
template <class C> __device__ __forceinline__ void cfma(C& acc, const C y, const C v) {
  acc.x = fmaT(y.x, v.x, fmaT(-y.y, v.y, acc.x));
  acc.y = fmaT(y.x, v.y, fmaT(y.y, v.x, acc.y));
}
// acc -= y * v (complex)
template <class C> __device__ __forceinline__ void cfms(C& acc, const C y, const C v) {
  acc.x = fmaT(-y.x, v.x, fmaT(y.y, v.y, acc.x));
  acc.y = fmaT(-y.x, v.y, fmaT(-y.y, v.x, acc.y));
}

// The per-element arithmetic of the forward epilogue and of the adjoint is
// written with explicit FMAs (no a*b + c left for the compiler to contract
// at its choice), so every kernel variant rounds it identically.
//   S = V conj(I):  P = Re V Re I + Im V Im I,  Q = Im V Re I - Re V Im I
template <class C> __device__ __forceinline__ C power_of(C v, C I) {
  return mkc(fmaT(v.x, I.x, v.y * I.y), fmaT(v.y, I.x, -(v.x * I.y)));
}
//   w = c conj(V) for c = ca + j cb
template <class C, class R> __device__ __forceinline__ C w_of(R ca, R cb, C v) {
  return mkc(fmaT(ca, v.x, cb * v.y), fmaT(cb, v.x, -(ca * v.y)));
}
//   h = conj(c) S + V z
template <class C> __device__ __forceinline__ C adj_h(C g0, C v, C z) {
  return mkc(g0.x + fmaT(v.x, z.x, -(v.y * z.y)), g0.y + fmaT(v.x, z.y, v.y * z.x));
}

// ---- cache policy of the optimiser state -------------------------------------
// Per iteration the adjoint pass streams the optimiser state (master theta,
// |V|, the moments, Q_calc at pv buses) through once, several times the L2's
// 129 MB at large batches.  It is read and written with the evict-first
// (streaming) policy, so that V and w, which the next pass gathers from, keep
// their L2 lines at normal priority.
#ifndef DPF_STREAM_HINTS
#define DPF_STREAM_HINTS 1
#endif
template <class T> __device__ __forceinline__ T ld_stream(const T* p) {
#if DPF_STREAM_HINTS
  return __ldcs(p);
#else
  return *p;
#endif
}
template <class T> __device__ __forceinline__ void st_stream(T* p, T v) {
#if DPF_STREAM_HINTS
  __stcs(p, v);
#else
  *p = v;
#endif
}

__device__ __forceinline__ Mom<float> mom_load(const Mom<float>* p) {
  const float4 t = ld_stream((const float4*)p);
  return Mom<float>{t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ void mom_store(Mom<float>* p, const Mom<float>& m) {
  st_stream((float4*)p, make_float4(m.m1, m.v1, m.m2, m.v2));
}
__device__ __forceinline__ Mom<double> mom_load(const Mom<double>* p) {
  const double2 a = ld_stream((const double2*)p), b = ld_stream((const double2*)p + 1);
  return Mom<double>{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void mom_store(Mom<double>* p, const Mom<double>& m) {
  st_stream((double2*)p, make_double2(m.m1, m.v1));
  st_stream((double2*)p + 1, make_double2(m.m2, m.v2));
}

// ---- programmatic dependent launch -------------------------------------------
// A kernel launched with programmatic stream serialisation may start while its
// predecessor drains.  pdl_wait() blocks until the predecessor grid has
// completed and its memory is visible; pdl_release() lets the successor be
// scheduled.  Both are no-ops for a kernel launched without the attribute.
// Everything before pdl_wait() may read only data no kernel of the iteration
// writes (Y_bus, bus types).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- master values ---------------------------------------------------------
// FP32 mode keeps theta and |V| as an unevaluated sum hi + lo of two floats
// (~48 significant bits) and updates them with an error-free two-sum, so the
// per-iteration path needs no FP64 instruction.
__device__ __forceinline__ double mval(float2 m) { return (double)m.x + (double)m.y; }
__device__ __forceinline__ double mval(double m) { return m; }
__device__ __forceinline__ float mwork(float2 m) { return m.x + m.y; }
__device__ __forceinline__ double mwork(double m) { return m; }

__device__ __forceinline__ float2 msub(float2 a, float d) {
  const float nd = -d;
  const float s = __fadd_rn(a.x, nd);
  const float bp = __fsub_rn(s, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bp)), __fsub_rn(nd, bp));
  const float lo = __fadd_rn(a.y, err);
  const float hi = __fadd_rn(s, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}
__device__ __forceinline__ double msub(double a, double d) { return a - d; }

template <class M> __device__ __forceinline__ M mfrom(double v);
template <> __device__ __forceinline__ float2 mfrom<float2>(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
template <> __device__ __forceinline__ double mfrom<double>(double v) { return v; }

// (theta, |V|) master pair of one element
__device__ __forceinline__ float2 ms_th(float4 s) { return make_float2(s.x, s.y); }
__device__ __forceinline__ float2 ms_vm(float4 s) { return make_float2(s.z, s.w); }
__device__ __forceinline__ float4 ms_make(float2 th, float2 vm) { return make_float4(th.x, th.y, vm.x, vm.y); }
__device__ __forceinline__ double ms_th(double2 s) { return s.x; }
__device__ __forceinline__ double ms_vm(double2 s) { return s.y; }
__device__ __forceinline__ double2 ms_make(double th, double vm) { return make_double2(th, vm); }

// V = |V| e^{j theta} in working precision.  FP32: sincos of the high word,
// first-order correction for the low word (|lo| <= 2^-24 |hi|).
__device__ __forceinline__ float2 volt(float2 th, float2 vm) {
  float s, c;
  sincosf(th.x, &s, &c);
  const float s2 = fmaf(th.y, c, s), c2 = fmaf(-th.y, s, c);
  const float m = vm.x + vm.y;
  return make_float2(m * c2, m * s2);
}
// The same, also returning the unit phasor u = e^{j theta} (V = |V| u); the
// refined FP32 adjoint's voltage.  The high word is first reduced to
// [-pi, pi] (Cody and Waite's reduction: k = rint(theta / 2 pi), theta - k 2 pi
// with 2 pi split into 6.28125, exact in 8 bits so that k * 6.28125 is exact,
// plus the float nearest 2 pi - 6.28125), then the SFU sine and cosine
// (__sincosf: absolute error below 4e-7 on [-pi, pi]).  u only scales the
// gradient and the step's voltage change, for which that suffices; the
// mismatch itself comes from the FP64 residual and dV.
__device__ __forceinline__ float2 volt(float2 th, float2 vm, float2& u) {
  float s, c;
  const float kk = rintf(th.x * 0.15915494f);  // 1 / (2 pi)
  const float red = fmaf(-kk, 1.93530718e-3f, fmaf(-kk, 6.28125f, th.x));
  __sincosf(red, &s, &c);
  u = make_float2(fmaf(-th.y, s, c), fmaf(th.y, c, s));
  const float m = vm.x + vm.y;
  return make_float2(m * u.x, m * u.y);
}
__device__ __forceinline__ double2 volt(double th, double vm) {
  double s, c;
  sincos(th, &s, &c);
  return make_double2(vm * c, vm * s);
}
// V in FP64 from a master value (the convergence test).
template <class M> __device__ __forceinline__ double2 volt64(M th, M vm) {
  double s, c;
  sincos(mval(th), &s, &c);
  const double m = mval(vm);
  return make_double2(m * c, m * s);
}



// ---- Y_bus views -----------------------------------------------------------
template <class R> struct YView;
template <> struct YView<float> {
  const int4* __restrict__ ent;  // {col, re bits, im bits, 0}
  __device__ __forceinline__ void get(int p, int& j, float2& y) const {
    const int4 e = __ldg(ent + p);
    j = e.x;
    y = make_float2(__int_as_float(e.y), __int_as_float(e.z));
  }
};
template <> struct YView<double> {
  const int32_t* __restrict__ col;
  const double2* __restrict__ val;
  __device__ __forceinline__ void get(int p, int& j, double2& y) const {
    j = __ldg(col + p);
    y = __ldg(val + p);
  }
};

// ---- thread -> (case, rows) map ------------------------------------------
struct Map {
  int k, row0, rstride, kl, rsub;
};
__device__ __forceinline__ Map thread_map(int lanes) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int rpw = 32 / lanes;
  Map mp;
  mp.kl = lane & (lanes - 1);
  mp.rsub = lane / lanes;
  mp.k = blockIdx.x * lanes + mp.kl;
  mp.row0 = (blockIdx.y * wpb + warp) * rpw + mp.rsub;
  mp.rstride = gridDim.y * wpb * rpw;
  return mp;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// Per-case max and sum over the CTA (convergence test), one atomic each.
__device__ __forceinline__ void case_max_sum_atomic(double mx, double sq, int lanes,
                                                    unsigned long long* omax, double* osum, int Kp) {
  __shared__ double rmax[32][32];
  __shared__ double rsum[32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int off = 16; off >= lanes; off >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    sq += __shfl_xor_sync(0xffffffffu, sq, off);
  }
  if (lane < lanes) { rmax[warp][lane] = mx; rsum[warp][lane] = sq; }
  __syncthreads();
  if (threadIdx.x < lanes) {
    double m = 0.0, s = 0.0;
    for (int w = 0; w < wpb; ++w) { m = fmax(m, rmax[w][threadIdx.x]); s += rsum[w][threadIdx.x]; }
    const int k = blockIdx.x * lanes + threadIdx.x;
    if (k < Kp) {
      atomic_max_nonneg(omax + k, m);
      if (s != 0.0) atomicAdd(osum + k, s);
    }
  }
}

// ---- row-block map and shared-memory Y_bus ----------------------------------
// CTA (bx, by) owns cases [bx*lanes, bx*lanes + lanes) and the contiguous bus
// rows [by*rpb, by*rpb + rpb).  Buses are RCM-ordered, so a row block is a
// compact patch of the grid: its Y_bus rows are staged once in shared memory
// (one coalesced copy) and the neighbour gathers of its warps hit the same
// cache lines.
struct BMap {
  int k, kl, rsub, i0, istride, r0, r1;
};
__device__ __forceinline__ BMap block_map(int lanes, int N, int rpb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int rpw = 32 / lanes;
  BMap mp;
  mp.kl = lane & (lanes - 1);
  mp.rsub = lane / lanes;
  mp.k = blockIdx.x * lanes + mp.kl;
  mp.r0 = blockIdx.y * rpb;
  mp.r1 = min(N, mp.r0 + rpb);
  mp.i0 = mp.r0 + warp * rpw + mp.rsub;
  mp.istride = wpb * rpw;
  return mp;
}

// Bytes of dynamic shared memory for a row block of `rows` rows and `nnz`
// padded entries, with the rows' bus types at the end (same formula on host
// and device).
__host__ __device__ __forceinline__ int ysmem_entries_end(int rows, int nnz, bool fp64) {
  const int rp = ((rows + 1) * 4 + 15) & ~15;
  return fp64 ? rp + ((nnz * 4 + 15) & ~15) + nnz * 16 : rp + nnz * 16;
}
__host__ __device__ __forceinline__ int ysmem_bytes(int rows, int nnz, bool fp64) {
  return ysmem_entries_end(rows, nnz, fp64) + ((rows + 15) & ~15);
}

// The row block's Y_bus rows and bus types in shared memory (a bus type
// decides which operands a row loads: read from here it costs no global
// round trip ahead of them).  Rows are padded to groups of four
// entries (a pad has weight 0 and points at the row's own bus, whose value
// the row's diagonal term reads anyway).  Each entry keeps its column as the
// element offset col * stride of the operand it gathers (stride: the case
// stride of the operand array, or of a shared-memory window), so a gather is
// one address computation from a per-thread base.  Offsets are 32-bit: the
// host keeps N * Kp below 2^32.
__device__ __forceinline__ int ysmem_pad_row(int pos) { return -pos - 1; }

template <class R> struct YSmem;
template <> struct YSmem<float> {
  const int* rp;
  const int4* ent;  // {offset, re bits, im bits, 0}
  const uint8_t* ty;
  __device__ __forceinline__ void stage(const int32_t* __restrict__ prp, const int32_t* __restrict__ ppos,
                                        const YView<float>& Y, const uint8_t* __restrict__ type, int r0, int r1,
                                        unsigned stride, unsigned char* sm) {
    const int nrow = max(0, r1 - r0);
    int* srp = (int*)sm;
    int4* sent = (int4*)(sm + (((nrow + 1) * 4 + 15) & ~15));
    const int base = nrow ? __ldg(prp + r0) : 0;
    const int cnt = nrow ? __ldg(prp + r1) - base : 0;
    for (int t = threadIdx.x; t <= nrow; t += blockDim.x) srp[t] = (nrow ? __ldg(prp + r0 + t) : 0) - base;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int pos = __ldg(ppos + base + t);
      int4 e;
      if (pos >= 0) {
        e = __ldg(Y.ent + pos);
        e.x = (int)((unsigned)e.x * stride);
      } else {
        e = make_int4((int)((unsigned)ysmem_pad_row(pos) * stride), 0, 0, 0);
      }
      sent[t] = e;
    }
    uint8_t* sty = sm + ysmem_entries_end(nrow, cnt, false);
    for (int t = threadIdx.x; t < nrow; t += blockDim.x) sty[t] = __ldg(type + r0 + t);
    __syncthreads();
    rp = srp - r0;  // index by global row
    ent = sent;
    ty = sty - r0;
  }
  __device__ __forceinline__ void get(int p, unsigned& o, float2& y) const {
    const int4 e = ent[p];
    o = (unsigned)e.x;
    y = make_float2(__int_as_float(e.y), __int_as_float(e.z));
  }
};
template <> struct YSmem<double> {
  const int* rp;
  const unsigned* off;
  const double2* val;
  const uint8_t* ty;
  __device__ __forceinline__ void stage(const int32_t* __restrict__ prp, const int32_t* __restrict__ ppos,
                                        const YView<double>& Y, const uint8_t* __restrict__ type, int r0, int r1,
                                        unsigned stride, unsigned char* sm) {
    const int nrow = max(0, r1 - r0);
    int* srp = (int*)sm;
    const int base = nrow ? __ldg(prp + r0) : 0;
    const int cnt = nrow ? __ldg(prp + r1) - base : 0;
    unsigned* soff = (unsigned*)(sm + (((nrow + 1) * 4 + 15) & ~15));
    double2* sval = (double2*)((unsigned char*)soff + ((cnt * 4 + 15) & ~15));
    for (int t = threadIdx.x; t <= nrow; t += blockDim.x) srp[t] = (nrow ? __ldg(prp + r0 + t) : 0) - base;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int pos = __ldg(ppos + base + t);
      if (pos >= 0) {
        soff[t] = (unsigned)__ldg(Y.col + pos) * stride;
        sval[t] = __ldg(Y.val + pos);
      } else {
        soff[t] = (unsigned)ysmem_pad_row(pos) * stride;
        sval[t] = make_double2(0.0, 0.0);
      }
    }
    uint8_t* sty = sm + ysmem_entries_end(nrow, cnt, true);
    for (int t = threadIdx.x; t < nrow; t += blockDim.x) sty[t] = __ldg(type + r0 + t);
    __syncthreads();
    rp = srp - r0;
    off = soff;
    val = sval;
    ty = sty - r0;
  }
  __device__ __forceinline__ void get(int p, unsigned& o, double2& y) const {
    o = off[p];
    y = val[p];
  }
};

// Single-case solves (one case per thread, Kp = 1): each Y_bus entry is used
// by exactly one thread, so staging the rows in shared memory buys no reuse
// and costs a round trip and a barrier per CTA.  This view reads the padded
// rows straight from global memory (entries {col, re bits, im bits, 0}, the
// pads pointing at their own row with weight 0, built per solve by
// k_pad_entries), so a CTA can own many rows and the grid one wave.
struct YDirect {
  const int* rp;      // padded row pointers, indexed by global row
  const int4* ent;
  const uint8_t* ty;
  __device__ __forceinline__ void get(int p, unsigned& o, float2& y) const {
    const int4 e = __ldg(ent + p);
    o = (unsigned)e.x;
    y = make_float2(__int_as_float(e.y), __int_as_float(e.z));
  }
  // Before the wait for the predecessor kernel (Y_bus does not change during
  // a solve): the thread's first row's entries and bus type toward L1, which
  // the staged view gets by staging before the wait.
  __device__ __forceinline__ void prefetch_row(int i, int r1) const {
    if (i >= r1) return;
    const int q0 = __ldg(rp + i);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ent + q0));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ty + i));
  }
};

// acc_row = sum_p Y[p] * X[offset(p)] over the row's padded entries [p0, p1)
// (X already points at this thread's case).  Four entries per step, so four
// independent gathers are in flight per thread; a pad adds an exact zero.
template <class R, class YS>
__device__ __forceinline__ typename Prec<R>::C row_spmv(const YS& ys, int p0, int p1,
                                                        const typename Prec<R>::C* __restrict__ X) {
  using C = typename Prec<R>::C;
  C a0 = mkc(R(0), R(0)), a1 = a0;
  for (int p = p0; p < p1; p += 4) {
    unsigned o[4];
    C y[4], x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ys.get(p + u, o[u], y[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = X[o[u]];
    cfma(a0, y[0], x[0]);
    cfma(a1, y[1], x[1]);
    cfma(a0, y[2], x[2]);
    cfma(a1, y[3], x[3]);
  }
  return mkc(a0.x + a1.x, a0.y + a1.y);
}

// ---- scheduler (one case) -------------------------------------------------
constexpr int SCHED_GROUP = 16;  // row blocks per group of the two-level loss sum

template <class R> struct SchedArgs {
  int Kp;
  int32_t* active;
  int32_t* iters;
  int32_t* status;
  const R* loss_part;  // [row blocks][Kp] the forward pass's loss partials
  R* grp_part;         // [groups][Kp] sums of SCHED_GROUP row blocks' partials (> 64 row blocks)
  unsigned int* grp_cnt;  // [tiles][groups] CTAs of a group done (reset by the group's last)
  unsigned int* mx32;  // FP32 max mismatch of the forward pass (or NULL)
  int32_t* cand;       // 1: the next FP64 test examines the case
  double gate;         // FP32 max mismatch below which the FP64 test runs (<= 0: always)
  double* lr;
  double* best;
  int32_t* bad;
  int32_t* cool;
  double* b1t;         // beta1^t, beta2^t of the last Adam step (running products)
  double* b2t;
  R* step_size;
  R* isbc2;
  int32_t* n_active;
  double inv_m, beta1, beta2, factor, threshold, min_lr, gamma, lr0;
  int sched, patience, cooldown, step_every, opt;
};

// Run once per active case per iteration, after the forward pass's loss and
// mismatch partials of that case are complete and before the adjoint pass:
//   1. the step terms of this iteration's update (step t + 1) from the current
//      rate (Adam: lr / (1 - beta1^(t+1)) and 1 / sqrt(1 - beta2^(t+1)));
//   2. the scheduler fed this iteration's loss (the loss of the iterate the
//      step is taken from), giving the rate of the next step.
// A non-finite loss stops the case as diverged before it steps.
template <class R>
__device__ __forceinline__ void sched_case(const SchedArgs<R>& a, int k, R lsum) {
  // every load is issued before the first store (one memory round trip: this
  // runs in the forward pass's tail, on its critical path)
  const int act = a.active[k];
  const unsigned mxu = a.mx32 ? __ldcg(a.mx32 + k) : 0u;
  const int it0 = a.iters[k];
  double lr = a.lr[k];
  const double b1p = a.b1t[k], b2p = a.b2t[k];
  const bool plateau = a.sched == SCHED_PLATEAU;
  double best = plateau ? a.best[k] : 0.0;
  int bad = plateau ? a.bad[k] : 0, cool = plateau ? a.cool[k] : 0;
  if (!act) return;
  const double L = (double)lsum * a.inv_m;
  if (a.mx32) {
    a.mx32[k] = 0u;
    a.cand[k] = (a.gate <= 0.0 || (double)__uint_as_float(mxu) <= a.gate) ? 1 : 0;
  }
  if (!isfinite(L)) {
    a.status[k] = CASE_DIVERGED;
    a.active[k] = 0;
    atomicSub(a.n_active, 1);
    return;
  }
  const int it = it0 + 1;  // number of the step about to be taken
  a.iters[k] = it;
  const double b1t = b1p * a.beta1, b2t = b2p * a.beta2;
  a.b1t[k] = b1t;
  a.b2t[k] = b2t;
  // (FP64 division and square root are slow on this GPU; FP32 runs only use
  // the step terms in FP32)
  if (a.opt == OPT_ADAM) {
    a.step_size[k] = (R)lr / (R(1) - (R)b1t);
    a.isbc2[k] = R(1) / sqrtT(R(1) - (R)b2t);
  } else {
    a.step_size[k] = (R)lr;
    a.isbc2[k] = R(1);
  }
  if (plateau) {
    if (L < best * (1.0 - a.threshold)) { best = L; bad = 0; }
    else bad += 1;
    if (cool > 0) { cool -= 1; bad = 0; }
    if (bad > a.patience) {
      const double nl = fmax(lr * a.factor, a.min_lr);
      if (lr - nl > 1e-8) lr = nl;
      cool = a.cooldown;
      bad = 0;
    }
    a.best[k] = best;
    a.bad[k] = bad;
    a.cool[k] = cool;
  } else if (a.sched == SCHED_STEP) {
    double gk = 1.0;  // gamma^(it / step_every) by repeated squaring (no pow: FP64 is slow here)
    double base = a.gamma;
    for (int e = it / a.step_every; e > 0; e >>= 1) {
      if (e & 1) gk *= base;
      base *= base;
    }
    lr = a.lr0 * gk;
  }
  a.lr[k] = lr;
}

// After a forward CTA's loss partials and mismatch atomics: the last CTA of its case tile
// (every CTA of the tile has counted itself after fencing its atomics) runs
// sched_case for the tile's cases and resets the tile counter.  Every thread
// of the CTA must call it.
template <class R>
__device__ __forceinline__ void tile_sched_grouped(const SchedArgs<R>& a, unsigned int* tile_cnt, int tile);

template <class R>
__device__ __forceinline__ void tile_sched(const SchedArgs<R>& a, unsigned int* tile_cnt, int tile) {
  if (gridDim.y > 64) {
    tile_sched_grouped(a, tile_cnt, tile);
    return;
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(tile_cnt + blockIdx.x, 1u);
    last = (prev == gridDim.y - 1);
    if (last) tile_cnt[blockIdx.x] = 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Each case's loss: its row blocks' partials summed in a fixed order, so
  // that a solve repeats bit for bit (an atomic sum's order varies between
  // runs); one thread per case.
  for (int c = threadIdx.x; c < tile; c += blockDim.x) {
    const int k = blockIdx.x * tile + c;
    if (k >= a.Kp) continue;
    R s = R(0);
    for (int yb = 0; yb < (int)gridDim.y; ++yb) s += __ldcg(a.loss_part + (size_t)yb * a.Kp + k);
    sched_case(a, k, s);
  }
}

// Many row blocks: two levels, each in a fixed order.  The last CTA of each
// group of SCHED_GROUP row blocks sums its group's partials (the groups' sums
// run in parallel in different CTAs); the last group of the case tile sums
// the groups' sums and takes the per-case step.
template <class R>
__device__ __forceinline__ void tile_sched_grouped(const SchedArgs<R>& a, unsigned int* tile_cnt, int tile) {
  __shared__ int lastg, last;
  const int ng = ((int)gridDim.y + SCHED_GROUP - 1) / SCHED_GROUP, g = (int)blockIdx.y / SCHED_GROUP;
  const int y0 = g * SCHED_GROUP, gsz = min(SCHED_GROUP, (int)gridDim.y - y0);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* c = a.grp_cnt + (size_t)blockIdx.x * ng + g;
    const unsigned prev = atomicAdd(c, 1u);
    lastg = (prev == (unsigned)gsz - 1);
    if (lastg) *c = 0u;
  }
  __syncthreads();
  if (!lastg) return;
  __threadfence();
  for (int c = threadIdx.x; c < tile; c += blockDim.x) {
    const int k = blockIdx.x * tile + c;
    if (k >= a.Kp) continue;
    R v[SCHED_GROUP];
#pragma unroll
    for (int u = 0; u < SCHED_GROUP; ++u) v[u] = u < gsz ? __ldcg(a.loss_part + (size_t)(y0 + u) * a.Kp + k) : R(0);
    R s = R(0);
#pragma unroll
    for (int u = 0; u < SCHED_GROUP; ++u) s += v[u];
    a.grp_part[(size_t)g * a.Kp + k] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(tile_cnt + blockIdx.x, 1u);
    last = (prev == (unsigned)ng - 1);
    if (last) tile_cnt[blockIdx.x] = 0u;
  }
  __syncthreads();
  if (!last) return;  // the same for every thread of the CTA
  __threadfence();
  // tpc threads per case (a power of two, tile * tpc <= blockDim.x <= 256)
  // take strided slices of the groups' sums, then a fixed tree: a single
  // case over hundreds of groups is summed by the whole CTA
  __shared__ R part[256];
  int tpc = 1;
  while (2 * tpc * tile <= (int)blockDim.x) tpc *= 2;
  const int per_pass = max(1, (int)blockDim.x / tpc);
  for (int c0 = 0; c0 < tile; c0 += per_pass) {
    const int c = c0 + (int)threadIdx.x / tpc, j = (int)threadIdx.x % tpc;
    const int k = blockIdx.x * tile + c;
    const bool mine = (int)threadIdx.x < per_pass * tpc && c < tile && k < a.Kp;
    R s = R(0);
    if (mine)
      for (int q = j; q < ng; q += tpc) s += __ldcg(a.grp_part + (size_t)q * a.Kp + k);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int step = tpc >> 1; step > 0; step >>= 1) {
      if (j < step) part[threadIdx.x] += part[threadIdx.x + step];
      __syncthreads();
    }
    if (mine && j == 0) sched_case(a, k, part[threadIdx.x]);
    __syncthreads();
  }
}

// n_active drops to 0 inside a forward pass when its scheduler stops the last
// running case as diverged: read it once per CTA so that all of a CTA's threads
// take the same branch (the caller's barriers follow).
__device__ __forceinline__ bool cta_idle(const int32_t* n_active) {
  __shared__ int idle;
  if (threadIdx.x == 0) idle = (n_active != nullptr && __ldcg(n_active) == 0);
  __syncthreads();
  return idle != 0;
}

// ---- arguments -------------------------------------------------------------
template <class R> struct IterArgs {
  using C = typename Prec<R>::C;
  using M = typename Prec<R>::M;
  int N, Kp, lanes, rpb;
  const int32_t* __restrict__ prp;   // padded row pointers (rows of 4k entries)
  const int32_t* __restrict__ ppos;  // padded slot -> CSR position, -(row+1) for a pad
  const int4* __restrict__ pent;     // padded entries in global memory (single-case direct view)
  YView<R> Y;
  const int32_t* wlo;  // per row block: first and last row its nonzeros reference
  const int32_t* whi;  //   (NULL: neighbour gathers read global memory)
  int ysmem;           // bytes of the staged Y rows (the V/W window follows)
  const uint8_t* __restrict__ type;
  C* V;
  C* W;
  R* qpv;    // Q_calc at pv buses (the rows k_adj cannot rebuild from w)
  typename Prec<R>::MS* ms;  // [N][Kp] master (theta, |V|)
  Mom<R>* os;                // [N][Kp] optimiser moments
  const R* pspec;
  const R* qspec;
  int spec_per_case;
  const int32_t* active;
  const int32_t* of;
  const int32_t* ot;
  const C* yff;
  const C* yft;
  const C* ytt;
  int has_outage;
  R* loss_part;        // [row blocks][Kp] per-CTA loss partials (solve loop; NULL: none)
  unsigned int* mx32;  // per-case max |dP|,|dQ| (float bits) or NULL
  const R* step_size;
  const R* isbc2;
  R beta1, beta2, eps, inv_m2, m_half;
  int opt;     // OPT_ADAM / OPT_SGD / OPT_RMSPROP
  R mom, alpha;  // SGD momentum, RMSprop smoothing
  const int32_t* n_active;
  // the per-case scheduler, run by the forward pass (solve loop only)
  SchedArgs<R> sc;
  unsigned int* tile_cnt;  // [case tiles] completion counters, NULL: no scheduler
  // mixed precision (DPF_MIXED): FP64 forward pass over FP64 voltages, FP32
  // adjoint and optimiser on the double-float master
  double2* V64m;           // [N][Kp] FP64 voltages (NULL: not mixed)
  YView<double> Y64;       // FP64 Y_bus values
  const double* pspec64;   // FP64 specified injections ([N][Kp] per case, or [N])
  const double* qspec64;
  const double2* yff64;    // FP64 N-1 blocks per case
  const double2* yft64;
  const double2* ytt64;
  double inv_m2_64;        // 2 / m in FP64
  // refined FP32 iterations (DPF_FP32R): V holds dV = V - V_ref, the change
  // of the voltages since the case's last FP64 test (or since 0 before its
  // first); vref = V_ref rounded to FP32, irf = (I_ref, f_ref) with I_ref the
  // FP64 current and f_ref the FP64 mismatch (dP, dQ; Q_calc at pv buses) at
  // V_ref, rounded to FP32.  NULL otherwise.
  const float2* vref;
  const float4* irf;
  // optional outputs (evaluation entry points); NULL in the solve loop
  C* sbuf;   // S_calc
  C* cbuf;   // c = (2/m)(dP + j dQ)
  R* gva;    // gradient mode of k_adj: write dL/dtheta, dL/d|V| instead of stepping
  R* gvm;
};

// Per-case sum and max over the CTA: the sum stored in this row block's slot
// of part_out ([row blocks][Kp]), the max by one atomic per case.  Every
// thread of the CTA must call it.
template <class R>
__device__ __forceinline__ void case_sum_max_atomic(R v, float mx, int lanes, R* part_out, unsigned int* max_out,
                                                    int Kp) {
  __shared__ R red[32][32];
  __shared__ float redm[32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int off = 16; off >= lanes; off >>= 1) {
    v += __shfl_xor_sync(0xffffffffu, v, off);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  }
  if (lane < lanes) {
    red[warp][lane] = v;
    redm[warp][lane] = mx;
  }
  __syncthreads();
  if (threadIdx.x < lanes) {
    R s = 0;
    float m = 0.f;
    for (int w = 0; w < wpb; ++w) {
      s += red[w][threadIdx.x];
      m = fmaxf(m, redm[w][threadIdx.x]);
    }
    const int k = blockIdx.x * lanes + threadIdx.x;
    if (k < Kp) {
      if (part_out) part_out[(size_t)blockIdx.y * Kp + k] = s;
      if (max_out && m > 0.f) atomicMax(max_out + k, __float_as_uint(m));
    }
  }
}

// Copy rows [lo, hi] of a case-minor array, restricted to this CTA's case
// tile, into shared memory: `per_row` 16-byte words per row, row-major.
// Coalesced 16-byte loads, all threads; ends with a barrier.
__device__ __forceinline__ void stage_window(const float4* __restrict__ src, unsigned row_words, unsigned base,
                                             int lo, int hi, int per_row, float4* __restrict__ dst) {
  const int n = (hi - lo + 1) * per_row;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int r = t / per_row, c = t - r * per_row;
    dst[t] = __ldg(src + (unsigned)(lo + r) * row_words + base + c);
  }
  __syncthreads();
}

// ---- forward: SpMV + power + mismatch + loss --------------------------------
// Refined FP32 epilogue (DPF_FP32R): with V = V_ref + dV and I = I_ref + Y dV,
//   S - S_spec = f_ref + dV conj(I_ref) + V conj(Y dV),
// so every FP32 rounding error scales with the change dV since the last FP64
// test (or with the small f_ref), not with |Y_ii| |V|.  Returns (dP, dQ) at
// pq buses, (dP, Q_calc) at pv buses; the caller masks by bus type.
__device__ __forceinline__ float2 refined_mismatch(float2 dv, float2 e, float2 vr, float4 rf, float2& v) {
  v = make_float2(vr.x + dv.x, vr.y + dv.y);
  const float2 t0 = power_of(dv, make_float2(rf.x, rf.y));
  const float2 t1 = power_of(v, e);
  return make_float2(rf.z + (t0.x + t1.x), rf.w + (t0.y + t1.y));
}

// The forward pass after its Y rows are in place (staged or direct).
template <class R, bool REF, class YS>
__device__ __forceinline__ void fwd_body(const IterArgs<R>& a, const YS& ys, const BMap& mp, bool staged,
                                         unsigned char* smem) {
  using C = typename Prec<R>::C;
  // the case's data in one round of independent loads, in flight during the
  // idle test (the outage arrays span Kp; an unused entry never matches a row)
  const int k = mp.k;
  const bool inb = k < a.Kp;
  const int act = inb ? a.active[k] : 0;
  int of = -1, ot = -1;  // (the outaged branch's block is loaded at its two rows)
  if (inb && a.has_outage) {
    of = a.of[k];
    ot = a.ot[k];
  }
  if (cta_idle(a.n_active)) {  // every CTA still counts itself for the scheduler
    if (a.tile_cnt) tile_sched(a.sc, a.tile_cnt, a.lanes);
    return;
  }
  const int wlo = staged ? a.wlo[blockIdx.y] : 0;
  C* vt = (C*)(smem + a.ysmem);
  if (staged) {
    constexpr int per_row = 32 * (int)sizeof(C) / 16;
    stage_window((const float4*)a.V, (unsigned)(a.Kp * sizeof(C) / 16), blockIdx.x * per_row, wlo,
                 a.whi[blockIdx.y], per_row, (float4*)vt);
  }
  const C* __restrict__ Vsh = vt - (size_t)wlo * 32 + (k & 31);
  const bool on = act != 0;
  R acc = 0;
  float mx = 0.f;
  if (on) {
    const size_t Kp = (size_t)a.Kp;
    const C* __restrict__ V = a.V;
    for (int i = mp.i0; i < mp.r1; i += mp.istride) {
      const size_t e = (size_t)i * Kp + k;
      const int ty = ys.ty[i];
      const size_t si = a.spec_per_case ? e : (size_t)i;
      // (refined mode: the gathered operand is dV, and I below is Y dV)
      const C xi = staged ? Vsh[(size_t)i * 32] : V[e];
      C I = staged ? row_spmv<R>(ys, ys.rp[i], ys.rp[i + 1], Vsh) : row_spmv<R>(ys, ys.rp[i], ys.rp[i + 1], V + k);
      if (i == of) {
        cfms(I, a.yff[k], xi);
        cfms(I, a.yft[k], V[(size_t)ot * Kp + k]);
      } else if (i == ot) {
        cfms(I, a.yft[k], V[(size_t)of * Kp + k]);
        cfms(I, a.ytt[k], xi);
      }
      C vi;
      R dP, dQ, Q;
      if constexpr (REF) {
        const float2 d = refined_mismatch(xi, I, ld_stream(a.vref + e), ld_stream(a.irf + e), vi);
        dP = (ty != BUS_SLACK) ? d.x : R(0);
        dQ = (ty == BUS_PQ) ? d.y : R(0);
        Q = d.y;
      } else {
        vi = xi;
        const R ps = a.pspec[si], qs = a.qspec[si];
        const C S = power_of(vi, I);
        Q = S.y;
        dP = (ty != BUS_SLACK) ? S.x - ps : R(0);
        dQ = (ty == BUS_PQ) ? Q - qs : R(0);
        if (a.sbuf) a.sbuf[e] = S;
      }
      const R ca = a.inv_m2 * dP, cb = a.inv_m2 * dQ;
      a.W[e] = w_of(ca, cb, vi);
      if (ty == BUS_PV) st_stream(a.qpv + e, Q);
      if (a.cbuf) a.cbuf[e] = mkc(ca, cb);
      acc = fmaT(dP, dP, fmaT(dQ, dQ, acc));
      const float am = fmaxf(fabsf((float)dP), fabsf((float)dQ));
      mx = (am != am) ? __int_as_float(0x7f800000) : fmaxf(mx, am);  // NaN -> +inf
    }
  }
  if (a.loss_part || a.mx32) case_sum_max_atomic(acc, mx, a.lanes, a.loss_part, a.mx32, a.Kp);
  if (a.tile_cnt) tile_sched(a.sc, a.tile_cnt, a.lanes);
}

template <class R, bool REF = false, bool DIRECT = false>
__global__ void __launch_bounds__(256, 5) k_fwd(IterArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BMap mp = block_map(a.lanes, a.N, a.rpb);
  if constexpr (DIRECT) {
    const YDirect ys{a.prp, a.pent, a.type};
    ys.prefetch_row(mp.i0, mp.r1);
    pdl_wait();
    pdl_release();
    fwd_body<R, REF>(a, ys, mp, false, smem);
  } else {
    // window of V in shared memory (lanes = 32: one 32-case line per row)
    const bool staged = a.wlo && a.lanes == 32 && mp.r0 < mp.r1;
    YSmem<R> ys;
    ys.stage(a.prp, a.ppos, a.Y, a.type, mp.r0, mp.r1, staged ? 32u : (unsigned)a.Kp, smem);
    pdl_wait();
    pdl_release();
    fwd_body<R, REF>(a, ys, mp, staged, smem);
  }
}

// conj(c_i) S_i rebuilt from w_i = c_i conj(V_i):  c = w V / |V|^2;
// P = P_spec + (m/2) Re c (pv, pq);  Q = Q_spec + (m/2) Im c (pq), or the
// forward pass's Q_calc at pv buses (c is real there).
template <class C, class R>
__device__ __forceinline__ C conj_c_s(C w, C v, int ty, R ps, R qs, R qpv, R m_half) {
  const R inv = div_step(R(1), fmaT(v.x, v.x, v.y * v.y));
  const R ca = fmaT(w.x, v.x, -(w.y * v.y)) * inv;
  const R cb = (ty == BUS_PQ) ? fmaT(w.x, v.y, w.y * v.x) * inv : R(0);
  const R P = fmaT(m_half, ca, ps);
  const R Q = (ty == BUS_PQ) ? fmaT(m_half, cb, qs) : qpv;
  return mkc(fmaT(ca, P, cb * Q), fmaT(ca, Q, -(cb * P)));
}

// ---- adjoint SpMV + gradient + Adam ----------------------------------------
// One optimiser step on a master value (Sec. 5.3's optimisers, PyTorch
// semantics).  step = lr (bias-corrected lr / (1 - beta1^t) for Adam), isb =
// 1 / sqrt(1 - beta2^t) (Adam); m, v are the per-element optimiser state.
// The amount subtracted from x is returned in d (the step, which the refined
// FP32 mode turns into the voltage change).
template <class R, class M>
__device__ __forceinline__ M opt_update(int opt, M x, R g, R& m, R& v, R b1, R b2, R step, R isb, R eps, R mom,
                                        R alpha, R& d) {
  if (opt == OPT_SGD) {
    m = (mom != R(0)) ? madd_step(mom, m, g) : g;
    d = step * m;
  } else if (opt == OPT_RMSPROP) {
    v = madd_step(alpha, v, ((R(1) - alpha) * g) * g);
    d = div_step(step * g, sqrt_step(v) + eps);
  } else {
    m = madd_step(b1, m, (R(1) - b1) * g);
    v = madd_step(b2, v, ((R(1) - b2) * g) * g);
    d = div_step(step * m, madd_step(sqrt_step(v), isb, eps));
  }
  return msub(x, d);
}
template <class R, class M>
__device__ __forceinline__ M opt_update(int opt, M x, R g, R& m, R& v, R b1, R b2, R step, R isb, R eps, R mom,
                                        R alpha) {
  R d;
  return opt_update(opt, x, g, m, v, b1, b2, step, isb, eps, mom, alpha, d);
}

// Refined FP32 mode: the change of V = |V| e^{j theta} over one step from the
// step itself, accurate relative to the change (no difference of two rounded
// voltages):  V' - V = u [|V| E + d|V| (1 + E)],  u = e^{j theta},
// E = e^{j dth} - 1 = (cos dth - 1) + j sin dth.  (Written with the unit
// phasor, it stays exact where |V| passes near 0.)  Optimiser steps are
// small: for |dth| <= 1/8 E comes from its Taylor series, cos x - 1 =
// -x^2/2 + x^4/24 - x^6/720 and sin x = x - x^3/6 + x^5/120 - x^7/5040
// (the first omitted terms are below 3e-11 relative), larger steps take
// E = 2 s (-s + j c) with (s, c) = (sin, cos)(dth / 2).
__device__ __forceinline__ float2 volt_change(float2 u, float m, float dth, float dm) {
  float ex, ey;
  if (fabsf(dth) <= 0.125f) {
    const float x2 = dth * dth;
    ex = 0.5f * x2 * fmaf(x2, fmaf(x2, -1.f / 360.f, 1.f / 12.f), -1.f);
    ey = dth * fmaf(x2, fmaf(x2, fmaf(x2, -1.f / 5040.f, 1.f / 120.f), -1.f / 6.f), 1.f);
  } else {
    float s, c;
    sincosf(0.5f * dth, &s, &c);
    ex = -2.f * s * s;
    ey = 2.f * s * c;
  }
  const float fx = fmaf(dm, 1.f + ex, m * ex), fy = fmaf(dm, ey, m * ey);
  return make_float2(fmaf(u.x, fx, -(u.y * fy)), fmaf(u.x, fy, u.y * fx));
}

#ifndef DPF_ADJ_ROWS
#define DPF_ADJ_ROWS 1
#endif

// One row of the adjoint pass for one case: operands, adjoint SpMV, update.
template <class R> struct AdjRow {
  using C = typename Prec<R>::C;
  using M = typename Prec<R>::M;
  bool live;  // row exists and is not the slack
  int i, ty;
  size_t e;
  C wi, vi, z;
  C dv;       // refined FP32 mode: dV = V - V_ref before the step
  C u;        // refined FP32 mode: e^{j theta} before the step (vi = |V| u)
  R ps, qs, qp, m1, v1, m2, v2;
  M th, vm;
};

template <class R, class YS, bool MIXED = false, bool REF = false>
__device__ __forceinline__ void adj_load(const IterArgs<R>& a, const YS& ys, AdjRow<R>& r, int i, int r1, int k,
                                         size_t Kp, bool grad_only) {
  r.live = false;
  if (i >= r1) return;
  r.i = i;
  r.e = (size_t)i * Kp + k;
  r.ty = ys.ty[i];
  if (r.ty == BUS_SLACK) {
    if (grad_only) { a.gva[r.e] = R(0); a.gvm[r.e] = R(0); }
    return;
  }
  r.live = true;
  const size_t e = r.e;
  r.wi = a.W[e];
  const size_t si = a.spec_per_case ? e : (size_t)i;
  r.ps = a.pspec[si];
  r.qs = a.qspec[si];
  r.qp = (r.ty == BUS_PV) ? ld_stream(a.qpv + e) : R(0);
  const typename Prec<R>::MS s = ld_stream(a.ms + e);
  r.th = ms_th(s);
  r.vm = ms_vm(s);
  if constexpr (MIXED) {  // the FP64 voltage, rounded for the FP32 adjoint
    const double2 v = a.V64m[e];
    r.vi = mkc((R)v.x, (R)v.y);
  } else if constexpr (REF) {  // the V buffer holds dV; V comes from the master (adj_finish)
    r.dv = a.V[e];
  } else {
    r.vi = a.V[e];  // = volt(th, vm), stored by the previous update (no second sincos)
  }
  r.m1 = r.v1 = r.m2 = r.v2 = R(0);
  if (!grad_only) {
    // full 16-byte accesses at pv buses too (their |V| halves pass through
    // unchanged): a half-written sector would cost a read-modify-write
    const Mom<R> o = mom_load(a.os + e);
    r.m1 = o.m1;
    r.v1 = o.v1;
    r.m2 = o.m2;
    r.v2 = o.v2;
  }
}

template <class R, class YS>
__device__ __forceinline__ void adj_gather(const IterArgs<R>& a, const YS& ys, AdjRow<R>& r, int k, size_t Kp,
                                           int of, int ot) {
  const int i = r.i;
  r.z = row_spmv<R>(ys, ys.rp[i], ys.rp[i + 1], a.W + k);
  if (i == of) {  // the outaged branch's block, loaded at its two rows
    cfms(r.z, a.yff[k], r.wi);
    cfms(r.z, a.yft[k], a.W[(size_t)ot * Kp + k]);
  } else if (i == ot) {
    cfms(r.z, a.yft[k], a.W[(size_t)of * Kp + k]);
    cfms(r.z, a.ytt[k], r.wi);
  }
}

template <class R, bool MIXED = false, bool REF = false>
__device__ __forceinline__ void adj_finish(const IterArgs<R>& a, AdjRow<R>& r, bool grad_only, R step, R isb, R b1,
                                           R b2, R eps) {
  using C = typename Prec<R>::C;
  const size_t e = r.e;
  if constexpr (REF) r.vi = volt(r.th, r.vm, r.u);  // (after the gather: fewer live registers across it)
  const C vi = r.vi, z = r.z;
  const C g0 = conj_c_s(r.wi, vi, r.ty, r.ps, r.qs, r.qp, a.m_half);
  const C h = adj_h(g0, vi, z);
  const R hr = h.x, hi = h.y;
  const R g_th = -hi;
  const R g_vm = (r.ty == BUS_PQ) ? div_step(hr, mwork(r.vm)) : R(0);
  if (grad_only) {
    a.gva[e] = g_th;
    a.gvm[e] = g_vm;
    return;
  }
  // optimiser step on theta (pv and pq buses) and on |V| (pq buses)
  R d_th = R(0), d_vm = R(0);
  const R vm_old = mwork(r.vm);
  r.th = opt_update(a.opt, r.th, g_th, r.m1, r.v1, b1, b2, step, isb, eps, a.mom, a.alpha, d_th);
  if (r.ty == BUS_PQ)
    r.vm = opt_update(a.opt, r.vm, g_vm, r.m2, r.v2, b1, b2, step, isb, eps, a.mom, a.alpha, d_vm);
  st_stream(a.ms + e, ms_make(r.th, r.vm));
  mom_store(a.os + e, Mom<R>{r.m1, r.v1, r.m2, r.v2});
  if constexpr (MIXED) {
    a.V64m[e] = volt64(r.th, r.vm);  // FP64 voltage from the master (FP64 sincos)
  } else if constexpr (REF) {        // dV grows by this step's change of V
    const float2 dd = volt_change(r.u, vm_old, -d_th, -d_vm);
    a.V[e] = make_float2(r.dv.x + dd.x, r.dv.y + dd.y);
  } else {
    a.V[e] = volt(r.th, r.vm);
  }
}

#ifndef DPF_ADJ_MINB
#define DPF_ADJ_MINB 4
#endif
// The adjoint pass after its Y rows are in place (staged or direct).
template <class R, bool MIXED, bool REF, class YS>
__device__ __forceinline__ void adj_body(const IterArgs<R>& a, const YS& ys, const BMap& mp) {
  using C = typename Prec<R>::C;
  // the case's data in one round of independent loads, in flight during the
  // idle test (the outage arrays span Kp; an unused entry never matches a row)
  const int k = mp.k;
  const bool inb = k < a.Kp;
  const bool grad_only = (a.gva != nullptr);
  const int act = inb ? a.active[k] : 0;
  int of = -1, ot = -1;
  if (inb && a.has_outage) {
    of = a.of[k];
    ot = a.ot[k];
  }
  R step = 0, isb = 1;
  if (inb && !grad_only) { step = a.step_size[k]; isb = a.isbc2[k]; }
  if (cta_idle(a.n_active) || !act) return;
  const R b1 = a.beta1, b2 = a.beta2, eps = a.eps;
  const size_t Kp = (size_t)a.Kp;
  const C* __restrict__ W = a.W;
  // DPF_ADJ_ROWS rows per warp per step: their loads and gathers are all
  // issued before any of them is consumed (more memory requests in flight)
  constexpr int NR = DPF_ADJ_ROWS;
  for (int i0 = mp.i0; i0 < mp.r1; i0 += NR * mp.istride) {
    AdjRow<R> rw[NR];
#pragma unroll
    for (int u = 0; u < NR; ++u)
      adj_load<R, YS, MIXED, REF>(a, ys, rw[u], i0 + u * mp.istride, mp.r1, k, Kp, grad_only);
#pragma unroll
    for (int u = 0; u < NR; ++u)
      if (rw[u].live) adj_gather(a, ys, rw[u], k, Kp, of, ot);
#pragma unroll
    for (int u = 0; u < NR; ++u)
      if (rw[u].live) adj_finish<R, MIXED, REF>(a, rw[u], grad_only, step, isb, b1, b2, eps);
  }
}

template <class R, bool MIXED = false, bool REF = false, bool DIRECT = false>
__global__ void __launch_bounds__(256, DPF_ADJ_MINB) k_adj(IterArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BMap mp = block_map(a.lanes, a.N, a.rpb);
  if constexpr (DIRECT) {
    const YDirect ys{a.prp, a.pent, a.type};
    ys.prefetch_row(mp.i0, mp.r1);
    pdl_wait();
    pdl_release();
    adj_body<R, MIXED, REF>(a, ys, mp);
  } else {
    YSmem<R> ys;
    ys.stage(a.prp, a.ppos, a.Y, a.type, mp.r0, mp.r1, (unsigned)a.Kp, smem);
    pdl_wait();
    pdl_release();
    adj_body<R, MIXED, REF>(a, ys, mp);
  }
}

// Padded entries of the direct view: slot p of the padded rows gets its
// CSR entry {col, re, im}, a pad {row, 0, 0} (weight 0 on its own row).
__global__ void k_pad_entries(const int32_t* __restrict__ ppos, const int4* __restrict__ ent, int n_pad,
                              int4* __restrict__ pent) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += gridDim.x * blockDim.x) {
    const int pos = ppos[p];
    int4 e;
    if (pos >= 0) {
      e = ent[pos];
      e.w = 0;
    } else {
      e = make_int4(ysmem_pad_row(pos), 0, 0, 0);
    }
    pent[p] = e;
  }
}

// ---- mixed precision forward pass (DPF_MIXED) -------------------------------
// The mismatch of a current I_i = sum_j Y_ij V_j that cancels terms of size
// |Y_ii| to a result of order 1 has an FP32 error of a few |Y_ii| 2^-24 --
// about 1e-5 p.u. on grids with short lines, above a 1e-6 p.u. target.  This
// pass reads FP64 voltages and FP64 Y_bus values and forms S, dP, dQ, the
// weights c and w = c conj(V) in FP64; it hands the FP32 adjoint w, Q_calc at
// pv buses and the loss partials in FP32 (the gradient needs no more: near
// convergence its error is relative to the small mismatch it is built from).
__global__ void __launch_bounds__(256, 4) k_fwd_mixed(IterArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BMap mp = block_map(a.lanes, a.N, a.rpb);
  YSmem<double> ys;
  ys.stage(a.prp, a.ppos, a.Y64, a.type, mp.r0, mp.r1, (unsigned)a.Kp, smem);
  pdl_wait();
  pdl_release();
  const int k = mp.k;
  const bool inb = k < a.Kp;
  const int act = inb ? a.active[k] : 0;
  int of = -1, ot = -1;
  double2 yff = make_double2(0.0, 0.0), yft = yff, ytt = yff;
  if (inb && a.has_outage) {
    of = a.of[k];
    ot = a.ot[k];
    yff = a.yff64[k];
    yft = a.yft64[k];
    ytt = a.ytt64[k];
  }
  if (cta_idle(a.n_active)) {  // every CTA still counts itself for the scheduler
    if (a.tile_cnt) tile_sched(a.sc, a.tile_cnt, a.lanes);
    return;
  }
  const double inv_m2 = a.inv_m2_64;
  double acc = 0.0;
  float mx = 0.f;
  if (act) {
    const size_t Kp = (size_t)a.Kp;
    const double2* __restrict__ V = a.V64m;
    for (int i = mp.i0; i < mp.r1; i += mp.istride) {
      const size_t e = (size_t)i * Kp + k;
      const int ty = ys.ty[i];
      const size_t si = a.spec_per_case ? e : (size_t)i;
      const double2 vi = V[e];
      const double ps = a.pspec64[si], qs = a.qspec64[si];
      double2 I = row_spmv<double>(ys, ys.rp[i], ys.rp[i + 1], V + k);
      if (i == of) {
        cfms(I, yff, vi);
        cfms(I, yft, V[(size_t)ot * Kp + k]);
      } else if (i == ot) {
        cfms(I, yft, V[(size_t)of * Kp + k]);
        cfms(I, ytt, vi);
      }
      const double2 S = power_of(vi, I);
      const double dP = (ty != BUS_SLACK) ? S.x - ps : 0.0;
      const double dQ = (ty == BUS_PQ) ? S.y - qs : 0.0;
      const double ca = inv_m2 * dP, cb = inv_m2 * dQ;
      const double2 w = w_of(ca, cb, vi);
      a.W[e] = make_float2((float)w.x, (float)w.y);
      if (ty == BUS_PV) st_stream(a.qpv + e, (float)S.y);
      acc = fma(dP, dP, fma(dQ, dQ, acc));
      const float am = (float)fmax(fabs(dP), fabs(dQ));
      mx = (am != am) ? __int_as_float(0x7f800000) : fmaxf(mx, am);  // NaN -> +inf
    }
  }
  if (a.loss_part || a.mx32) case_sum_max_atomic((float)acc, mx, a.lanes, a.loss_part, a.mx32, a.Kp);
  if (a.tile_cnt) tile_sched(a.sc, a.tile_cnt, a.lanes);
}

// FP64 voltages from the double-float master (mixed precision set-up).
__global__ void k_mixed_v64(const float4* __restrict__ ms, double2* __restrict__ v, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float4 s = ms[e];
    v[e] = volt64(ms_th(s), ms_vm(s));
  }
}

// ---- two cases per thread (FP32 solve loop, batches of >= 64 cases) --------
// Thread t of CTA bx handles the adjacent cases k0 = 2 (bx*32 + lane) and
// k0 + 1: the row's Y entries, bus type and address arithmetic serve both,
// and every per-element access is one 16-byte (two-case) load or store.
struct Pair {
  int k0;
  bool on0, on1;
  int of0, ot0, of1, ot1;
};

// One round of independent loads: k0 is even and k0 + 1 < Kp (Kp is a
// multiple of 64 here), so each two-case access is one aligned 8-byte load.
// The outage rows are read whether or not a case has an outage (the arrays
// span Kp; an unused entry never matches a row).  The outaged branch's 2x2
// block is not kept in registers across the row loop: the two rows of a case
// that need it load it there (out_block).
__device__ __forceinline__ Pair load_pair(const IterArgs<float>& a, int k0) {
  Pair q;
  q.k0 = k0;
  const int2 act = *(const int2*)(a.active + k0);
  q.of0 = q.ot0 = q.of1 = q.ot1 = -1;
  if (a.has_outage) {
    const int2 of = *(const int2*)(a.of + k0), ot = *(const int2*)(a.ot + k0);
    q.of0 = of.x; q.of1 = of.y;
    q.ot0 = ot.x; q.ot1 = ot.y;
  }
  q.on0 = act.x != 0;
  q.on1 = act.y != 0;
  return q;
}

// acc -= the outaged branch's block applied at row i of case k (i is that
// case's from-bus `of` or to-bus `ot`): x_i is the case's own operand at row
// i, x_o its operand at the branch's other end.
__device__ __forceinline__ void out_block(const IterArgs<float>& a, int k, bool from, float2 x_i, float2 x_o,
                                          float2& acc) {
  if (from) {  // row f: Y_ff x_f + Y_ft x_t
    cfms(acc, a.yff[k], x_i);
    cfms(acc, a.yft[k], x_o);
  } else {     // row t: Y_tf x_f + Y_tt x_t (Y_tf = Y_ft)
    cfms(acc, a.yft[k], x_o);
    cfms(acc, a.ytt[k], x_i);
  }
}

// sum_p Y[p] X[offset(p)] for two adjacent cases (X as float4 pairs, already
// pointing at this thread's pair); padded rows as in row_spmv.
__device__ __forceinline__ void row_spmv2(const YSmem<float>& ys, int p0, int p1, const float4* __restrict__ X,
                                          float2& r0, float2& r1) {
  // two accumulators per case, alternating like row_spmv: the same sums
  float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
  for (int p = p0; p < p1; p += 4) {
    unsigned o[4];
    float2 y[4];
    float4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ys.get(p + u, o[u], y[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = X[o[u]];
    cfma(a0, y[0], make_float2(x[0].x, x[0].y));
    cfma(b0, y[0], make_float2(x[0].z, x[0].w));
    cfma(a1, y[1], make_float2(x[1].x, x[1].y));
    cfma(b1, y[1], make_float2(x[1].z, x[1].w));
    cfma(a0, y[2], make_float2(x[2].x, x[2].y));
    cfma(b0, y[2], make_float2(x[2].z, x[2].w));
    cfma(a1, y[3], make_float2(x[3].x, x[3].y));
    cfma(b1, y[3], make_float2(x[3].z, x[3].w));
  }
  r0 = make_float2(a0.x + a1.x, a0.y + a1.y);
  r1 = make_float2(b0.x + b1.x, b0.y + b1.y);
}

// Per-case sum (into this row block's slot of part_out) and max (one atomic)
// for two cases per thread.
__device__ __forceinline__ void pair_sum_max_atomic(float s0, float s1, float m0, float m1, float* part_out,
                                                    unsigned int* max_out, int Kp) {
  __shared__ float rs[8][64];
  __shared__ float rm[8][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  rs[warp][2 * lane] = s0;
  rs[warp][2 * lane + 1] = s1;
  rm[warp][2 * lane] = m0;
  rm[warp][2 * lane + 1] = m1;
  __syncthreads();
  if (threadIdx.x < 64) {
    float s = 0.f, m = 0.f;
    for (int w = 0; w < wpb; ++w) {
      s += rs[w][threadIdx.x];
      m = fmaxf(m, rm[w][threadIdx.x]);
    }
    const int k = blockIdx.x * 64 + threadIdx.x;
    if (k < Kp) {
      if (part_out) part_out[(size_t)blockIdx.y * Kp + k] = s;
      if (max_out && m > 0.f) atomicMax(max_out + k, __float_as_uint(m));
    }
  }
}

// Forward epilogue of one case (the same arithmetic as k_fwd).
__device__ __forceinline__ void fwd_epilogue(float2 vi, float2 I, int ty, float ps, float qs, float inv_m2,
                                             float2& w, float& q, float& acc, float& mx) {
  const float2 S = power_of(vi, I);
  const float P = S.x, Q = S.y;
  const float dP = (ty != BUS_SLACK) ? P - ps : 0.f;
  const float dQ = (ty == BUS_PQ) ? Q - qs : 0.f;
  const float ca = inv_m2 * dP, cb = inv_m2 * dQ;
  w = w_of(ca, cb, vi);
  q = Q;
  acc = fmaf(dP, dP, fmaf(dQ, dQ, acc));
  const float am = fmaxf(fabsf(dP), fabsf(dQ));
  mx = (am != am) ? __int_as_float(0x7f800000) : fmaxf(mx, am);
}

// The same for the refined FP32 mode: dv = dV, e = Y dV (see refined_mismatch).
__device__ __forceinline__ void fwd_epilogue_ref(float2 dv, float2 e, float2 vr, float4 rf, int ty, float inv_m2,
                                                 float2& w, float& q, float& acc, float& mx) {
  float2 v;
  const float2 d = refined_mismatch(dv, e, vr, rf, v);
  const float dP = (ty != BUS_SLACK) ? d.x : 0.f;
  const float dQ = (ty == BUS_PQ) ? d.y : 0.f;
  const float ca = inv_m2 * dP, cb = inv_m2 * dQ;
  w = w_of(ca, cb, v);
  q = d.y;
  acc = fmaf(dP, dP, fmaf(dQ, dQ, acc));
  const float am = fmaxf(fabsf(dP), fabsf(dQ));
  mx = (am != am) ? __int_as_float(0x7f800000) : fmaxf(mx, am);
}

#ifndef DPF_FWD2_MINB
#define DPF_FWD2_MINB 4
#endif
template <bool REF = false>
__global__ void __launch_bounds__(256, DPF_FWD2_MINB) k_fwd2(IterArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int r0 = blockIdx.y * a.rpb, r1 = min(a.N, r0 + a.rpb);
  const unsigned hKp = (unsigned)a.Kp >> 1;
  YSmem<float> ys;
  ys.stage(a.prp, a.ppos, a.Y, a.type, r0, r1, (a.wlo && r0 < r1) ? 32u : hKp, smem);
  pdl_wait();
  pdl_release();
  const int k0 = 2 * (blockIdx.x * 32 + lane);
  const Pair q = load_pair(a, k0);  // in flight during the idle test
  if (cta_idle(a.n_active)) {  // every CTA still counts itself for the scheduler
    if (a.tile_cnt) tile_sched(a.sc, a.tile_cnt, 64);
    return;
  }
  const unsigned h0 = (unsigned)k0 >> 1;
  // this block's window of V (the rows its nonzeros reference), one
  // 512-byte line of 64 cases per row
  const int wlo = (a.wlo && r0 < r1) ? a.wlo[blockIdx.y] : 0;
  float4* vt = (float4*)(smem + a.ysmem);
  if (a.wlo && r0 < r1) stage_window((const float4*)a.V, hKp, blockIdx.x * 32, wlo, a.whi[blockIdx.y], 32, vt);
  const float4* __restrict__ Vs = vt - (size_t)wlo * 32 + lane;  // Vs[j * 32]: row j, this thread's pair
  float acc0 = 0.f, acc1 = 0.f, mx0 = 0.f, mx1 = 0.f;
  if (q.on0 || q.on1) {
    const float4* __restrict__ V = (const float4*)a.V;
    float4* W = (float4*)a.W;
    for (int i = r0 + warp; i < r1; i += wpb) {
      const unsigned e = (unsigned)i * hKp + h0;  // pair index
      const int ty = ys.ty[i];
      const float4 v = a.wlo ? Vs[(size_t)i * 32] : V[e];  // (refined mode: dV)
      float ps0 = 0.f, ps1 = 0.f, qs0 = 0.f, qs1 = 0.f;
      float4 vr, rf0, rf1;
      if constexpr (REF) {
        vr = ld_stream((const float4*)a.vref + e);
        rf0 = ld_stream(a.irf + 2 * (size_t)e);
        rf1 = ld_stream(a.irf + 2 * (size_t)e + 1);
      } else if (a.spec_per_case) {
        const float2 pp = ((const float2*)a.pspec)[e], qq = ((const float2*)a.qspec)[e];
        ps0 = pp.x; ps1 = pp.y; qs0 = qq.x; qs1 = qq.y;
      } else {
        ps0 = ps1 = a.pspec[i];
        qs0 = qs1 = a.qspec[i];
      }
      float2 I0, I1;
      row_spmv2(ys, ys.rp[i], ys.rp[i + 1], a.wlo ? Vs : V + h0, I0, I1);
      const float2 vi0 = make_float2(v.x, v.y), vi1 = make_float2(v.z, v.w);
      if (i == q.of0 || i == q.ot0) {
        const float4 t = V[(unsigned)(i == q.of0 ? q.ot0 : q.of0) * hKp + h0];
        out_block(a, q.k0, i == q.of0, vi0, make_float2(t.x, t.y), I0);
      }
      if (i == q.of1 || i == q.ot1) {
        const float4 t = V[(unsigned)(i == q.of1 ? q.ot1 : q.of1) * hKp + h0];
        out_block(a, q.k0 + 1, i == q.of1, vi1, make_float2(t.z, t.w), I1);
      }
      float2 w0, w1;
      float q0, q1;
      if constexpr (REF) {
        fwd_epilogue_ref(vi0, I0, make_float2(vr.x, vr.y), rf0, ty, a.inv_m2, w0, q0, acc0, mx0);
        fwd_epilogue_ref(vi1, I1, make_float2(vr.z, vr.w), rf1, ty, a.inv_m2, w1, q1, acc1, mx1);
      } else {
        fwd_epilogue(vi0, I0, ty, ps0, qs0, a.inv_m2, w0, q0, acc0, mx0);
        fwd_epilogue(vi1, I1, ty, ps1, qs1, a.inv_m2, w1, q1, acc1, mx1);
      }
      W[e] = make_float4(w0.x, w0.y, w1.x, w1.y);
      if (ty == BUS_PV) st_stream((float2*)a.qpv + e, make_float2(q0, q1));
    }
    if (!q.on0) { acc0 = 0.f; mx0 = 0.f; }
    if (!q.on1) { acc1 = 0.f; mx1 = 0.f; }
  }
  pair_sum_max_atomic(acc0, acc1, mx0, mx1, a.loss_part, a.mx32, a.Kp);
  if (a.tile_cnt) tile_sched(a.sc, a.tile_cnt, 64);
}


template <bool REF = false>
__global__ void __launch_bounds__(256, 4) k_adj2(IterArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int r0 = blockIdx.y * a.rpb, r1 = min(a.N, r0 + a.rpb);
  YSmem<float> ys;
  ys.stage(a.prp, a.ppos, a.Y, a.type, r0, r1, (unsigned)a.Kp >> 1, smem);
  pdl_wait();
  pdl_release();
  const int k0 = 2 * (blockIdx.x * 32 + lane);
  const Pair q = load_pair(a, k0);
  const float2 st = *(const float2*)(a.step_size + k0), ib = *(const float2*)(a.isbc2 + k0);
  if (cta_idle(a.n_active) || !(q.on0 || q.on1)) return;
  const float st0 = st.x, st1 = st.y, ib0 = ib.x, ib1 = ib.y;
  const float b1 = a.beta1, b2 = a.beta2, eps = a.eps;
  const unsigned hKp = (unsigned)a.Kp >> 1, h0 = (unsigned)k0 >> 1;
  const float4* __restrict__ W = (const float4*)a.W;
  for (int i = r0 + warp; i < r1; i += wpb) {
    const int ty = ys.ty[i];
    if (ty == BUS_SLACK) continue;
    const unsigned e = (unsigned)i * hKp + h0;
    // this element's operands first: they do not depend on the gather chain
    const float4 wi = W[e];
    float ps0, ps1, qs0, qs1;
    if (a.spec_per_case) {
      const float2 pp = ((const float2*)a.pspec)[e], qq = ((const float2*)a.qspec)[e];
      ps0 = pp.x; ps1 = pp.y; qs0 = qq.x; qs1 = qq.y;
    } else {
      ps0 = ps1 = a.pspec[i];
      qs0 = qs1 = a.qspec[i];
    }
    const float2 qp = (ty == BUS_PV) ? ld_stream((const float2*)a.qpv + e) : make_float2(0.f, 0.f);
    const float4 s0 = ld_stream(a.ms + 2 * (size_t)e), s1 = ld_stream(a.ms + 2 * (size_t)e + 1);
    // current V of both cases (no second sincos); refined mode: dV (V from the master)
    const float4 vv4 = ((const float4*)a.V)[e];
    Mom<float> o0 = mom_load(a.os + 2 * (size_t)e), o1 = mom_load(a.os + 2 * (size_t)e + 1);
    float2 z0, z1;
    row_spmv2(ys, ys.rp[i], ys.rp[i + 1], W + h0, z0, z1);
    if (i == q.of0 || i == q.ot0) {
      const float4 t = W[(unsigned)(i == q.of0 ? q.ot0 : q.of0) * hKp + h0];
      out_block(a, q.k0, i == q.of0, make_float2(wi.x, wi.y), make_float2(t.x, t.y), z0);
    }
    if (i == q.of1 || i == q.ot1) {
      const float4 t = W[(unsigned)(i == q.of1 ? q.ot1 : q.of1) * hKp + h0];
      out_block(a, q.k0 + 1, i == q.of1, make_float2(wi.z, wi.w), make_float2(t.z, t.w), z1);
    }
    float2 th0 = ms_th(s0), th1 = ms_th(s1);
    float2 vm0 = ms_vm(s0), vm1 = ms_vm(s1);
    float2 u0, u1, v0, v1;
    if constexpr (REF) {
      v0 = volt(ms_th(s0), ms_vm(s0), u0);
      v1 = volt(ms_th(s1), ms_vm(s1), u1);
    } else {
      v0 = make_float2(vv4.x, vv4.y);
      v1 = make_float2(vv4.z, vv4.w);
    }
    const float2 g0 = conj_c_s(make_float2(wi.x, wi.y), v0, ty, ps0, qs0, qp.x, a.m_half);
    const float2 g1 = conj_c_s(make_float2(wi.z, wi.w), v1, ty, ps1, qs1, qp.y, a.m_half);
    const float2 h0 = adj_h(g0, v0, z0), h1 = adj_h(g1, v1, z1);
    const float hr0 = h0.x, hi0 = h0.y, hr1 = h1.x, hi1 = h1.y;
    // optimiser step on theta (pv and pq buses); an inactive case keeps its state
    float dth0 = 0.f, dth1 = 0.f, dvm0 = 0.f, dvm1 = 0.f;
    const float m0 = mwork(vm0), m1 = mwork(vm1);
    if (q.on0) th0 = opt_update(a.opt, th0, -hi0, o0.m1, o0.v1, b1, b2, st0, ib0, eps, a.mom, a.alpha, dth0);
    if (q.on1) th1 = opt_update(a.opt, th1, -hi1, o1.m1, o1.v1, b1, b2, st1, ib1, eps, a.mom, a.alpha, dth1);
    if (ty == BUS_PQ) {  // and on |V| (pq buses)
      if (q.on0) vm0 = opt_update(a.opt, vm0, div_step(hr0, m0), o0.m2, o0.v2, b1, b2, st0, ib0, eps, a.mom,
                                  a.alpha, dvm0);
      if (q.on1) vm1 = opt_update(a.opt, vm1, div_step(hr1, m1), o1.m2, o1.v2, b1, b2, st1, ib1, eps, a.mom,
                                  a.alpha, dvm1);
    }
    st_stream(a.ms + 2 * (size_t)e, ms_make(th0, vm0));
    st_stream(a.ms + 2 * (size_t)e + 1, ms_make(th1, vm1));
    mom_store(a.os + 2 * (size_t)e, o0);
    mom_store(a.os + 2 * (size_t)e + 1, o1);
    if constexpr (REF) {  // dV grows by this step's change of V (an inactive case has a zero step)
      const float2 d0 = volt_change(u0, m0, -dth0, -dvm0);
      const float2 d1 = volt_change(u1, m1, -dth1, -dvm1);
      ((float4*)a.V)[e] = make_float4(vv4.x + d0.x, vv4.y + d0.y, vv4.z + d1.x, vv4.w + d1.y);
    } else {
      const float2 n0 = q.on0 ? volt(th0, vm0) : v0, n1 = q.on1 ? volt(th1, vm1) : v1;
      ((float4*)a.V)[e] = make_float4(n0.x, n0.y, n1.x, n1.y);
    }
  }
}

// ---- FP64 convergence test --------------------------------------------------
// Whether the test examines active case k: every case without a gate (cand
// NULL), else the cases the gate admitted, plus -- with full_every > 0 (the
// refined FP32 mode, ~100 steps) -- every case whose step count is a
// multiple of full_every, so that no case runs on one reference for long
// (with large steps its FP32 bookkeeping of dV drifts by a few 1e-9 per
// step).  The three test kernels take the same decision from the same inputs.
__device__ __forceinline__ bool examined(const int32_t* cand, const int32_t* iters, int full_every, int k) {
  return !cand || cand[k] || (full_every > 0 && iters[k] % full_every == 0);
}

template <class M> struct Check64Args {
  int N, Kp, lanes, all_cases;
  const int32_t* __restrict__ rp;
  const int32_t* __restrict__ col;
  const double2* __restrict__ val;
  const uint8_t* __restrict__ type;
  const typename std::conditional<std::is_same<M, float2>::value, float4, double2>::type* ms;  // master pairs
  double2* V64;
  const double* pspec;
  const double* qspec;
  int spec_per_case;
  const int32_t* active;
  const int32_t* cand;  // NULL: every active case; else only cases with cand[k] = 1
  const int32_t* iters;  // per-case step counts (full_every)
  int full_every;        // > 0: also every case whose step count is a multiple of this
  const int32_t* of;
  const int32_t* ot;
  const double2* yff;
  const double2* yft;
  const double2* ytt;
  int has_outage;
  unsigned long long* maxmis;
  double* loss64;
  const int32_t* n_active;
  // refined FP32 mode, tests inside the loop: every examined case restarts its
  // FP32 iterations from this test's FP64 values (vref, irf: see IterArgs;
  // dv, the V buffer of the iterations, is set to 0)
  int refresh;
  float2* vref;
  float4* irf;
  float2* dv;
};

// V64 = |V| e^{j theta} from the master state (FP64 sincos).
template <class M>
__global__ void __launch_bounds__(1024) k_volt64(Check64Args<M> a) {
  pdl_wait();
  pdl_release();
  if (!a.all_cases && *a.n_active == 0) return;
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  if (k >= a.Kp || !(a.all_cases || (a.active[k] && examined(a.cand, a.iters, a.full_every, k)))) return;
  for (int i = mp.row0; i < a.N; i += mp.rstride) {
    const size_t e = (size_t)i * a.Kp + k;
    const auto s = a.ms[e];
    a.V64[e] = volt64(ms_th(s), ms_vm(s));
  }
}

template <class M>
__global__ void __launch_bounds__(1024) k_check64(Check64Args<M> a) {
  pdl_wait();
  pdl_release();
  if (!a.all_cases && *a.n_active == 0) return;
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  const bool on = (k < a.Kp) && (a.all_cases || (a.active[k] && examined(a.cand, a.iters, a.full_every, k)));
  double mx = 0.0, sq = 0.0;
  if (on) {
    int of = -1, ot = -1;
    double2 yff = make_double2(0, 0), yft = yff, ytt = yff;
    if (a.has_outage) {
      of = a.of[k];
      ot = a.ot[k];
      if (of >= 0) { yff = a.yff[k]; yft = a.yft[k]; ytt = a.ytt[k]; }
    }
    const size_t Kp = (size_t)a.Kp;
    const double2* __restrict__ V = a.V64;
    for (int i = mp.row0; i < a.N; i += mp.rstride) {
      const size_t e = (size_t)i * Kp + k;
      double2 I = make_double2(0.0, 0.0);
      const int p1 = __ldg(a.rp + i + 1);
      for (int p = __ldg(a.rp + i); p < p1; ++p)
        cfma(I, __ldg(a.val + p), V[(size_t)__ldg(a.col + p) * Kp + k]);
      const double2 vi = V[e];
      if (i == of) {
        cfms(I, yff, vi);
        cfms(I, yft, V[(size_t)ot * Kp + k]);
      } else if (i == ot) {
        cfms(I, yft, V[(size_t)of * Kp + k]);
        cfms(I, ytt, vi);
      }
      const double P = vi.x * I.x + vi.y * I.y;
      const double Q = vi.y * I.x - vi.x * I.y;
      const int ty = __ldg(a.type + i);
      const size_t si = a.spec_per_case ? e : (size_t)i;
      const double dP = (ty != BUS_SLACK) ? P - a.pspec[si] : 0.0;
      const double dQ = (ty == BUS_PQ) ? Q - a.qspec[si] : 0.0;
      // a NaN mismatch is recorded as +inf so that it survives the max reduction
      const double am = (isnan(dP) || isnan(dQ)) ? __longlong_as_double(0x7ff0000000000000LL)
                                                 : fmax(fabs(dP), fabs(dQ));
      mx = fmax(mx, am);
      sq += dP * dP + dQ * dQ;
      if (a.refresh) {
        a.vref[e] = make_float2((float)vi.x, (float)vi.y);
        a.irf[e] = make_float4((float)I.x, (float)I.y, (float)dP, (float)((ty == BUS_PV) ? Q : dQ));
        a.dv[e] = make_float2(0.f, 0.f);
      }
    }
  }
  case_max_sum_atomic(mx, sq, a.lanes, a.maxmis, a.loss64, a.Kp);
}

// Apply a convergence test (single CTA): stop converged cases, record their
// mismatch, reset the accumulators and recount the active cases.  With
// `final_pass` every real case gets its outputs and final status.
struct ApplyArgs {
  int K, Kp, final_pass;
  double tol, inv_m;
  int32_t* active;
  const int32_t* cand;
  const int32_t* iters;
  int full_every;
  int32_t* status;
  unsigned long long* maxmis;
  double* loss64;
  double* out_max;
  double* out_loss;
  int32_t* n_active;
};

__global__ void k_apply(ApplyArgs a) {
  __shared__ int cnt[32];
  pdl_wait();
  pdl_release();
  int c = 0;
  for (int k = threadIdx.x; k < a.Kp; k += blockDim.x) {
    if (k < a.K) {
      const double mx = __longlong_as_double((long long)a.maxmis[k]);
      const double L = a.loss64[k] * a.inv_m;
      if (a.final_pass) {
        a.out_max[k] = mx;
        a.out_loss[k] = L;
        if (a.active[k]) a.status[k] = (mx <= a.tol) ? CASE_CONVERGED : CASE_MAX_ITER;
        a.active[k] = 0;
      } else if (a.active[k] && examined(a.cand, a.iters, a.full_every, k) && mx <= a.tol) {
        a.active[k] = 0;
        a.status[k] = CASE_CONVERGED;
        a.out_max[k] = mx;
        a.out_loss[k] = L;
      }
      c += a.active[k];
    }
    a.maxmis[k] = 0ULL;
    a.loss64[k] = 0.0;
  }
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += cnt[w];
    *a.n_active = s;
  }
}

// Initial reference of the refined FP32 mode: V_ref = 0, I_ref = 0, so the
// first iterations evaluate f = V conj(Y V) - S_spec like plain FP32 ones (the
// V buffer holds dV = V) until the case's first FP64 test.  f_ref = -S_spec
// (pv buses: Q_calc(V_ref) = 0).  p, q: FP32 specification, [N][Kp] if
// per_case, else [N].
__global__ void k_ref_init(const uint8_t* __restrict__ type, const float* __restrict__ p,
                           const float* __restrict__ q, int per_case, int Kp, size_t n, float2* __restrict__ vref,
                           float4* __restrict__ irf) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Kp);
    const int ty = type[i];
    const size_t si = per_case ? e : (size_t)i;
    vref[e] = make_float2(0.f, 0.f);
    irf[e] = make_float4(0.f, 0.f, (ty != BUS_SLACK) ? -p[si] : 0.f, (ty == BUS_PQ) ? -q[si] : 0.f);
  }
}

// Re-activate the first K of Kp cases (a final convergence pass deactivates all).
__global__ void k_activate(int32_t* __restrict__ active, int K, int Kp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < Kp) active[k] = (k < K) ? 1 : 0;
}

// ---- set-up / tear-down ----------------------------------------------------
// Tiled transpose of a case-major [K][N] user-order FP64 array into the
// case-minor internal layout [N][Kp] (row iperm[u] for user bus u).
__global__ void k_to_internal(const double* __restrict__ src, double* __restrict__ dst, int K, int N,
                              int Kp, const int32_t* __restrict__ iperm) {
  __shared__ double tile[32][33];
  const int u0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, u = u0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && u < N) ? src[(size_t)k * N + u] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int u = u0 + r, k = k0 + threadIdx.x;
    if (u < N && k < K) dst[(size_t)iperm[u] * Kp + k] = tile[threadIdx.x][r];
  }
}

// Inverse of k_to_internal.
__global__ void k_to_user(const double* __restrict__ src, double* __restrict__ dst, int K, int N, int Kp,
                          const int32_t* __restrict__ iperm) {
  __shared__ double tile[32][33];
  const int u0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int u = u0 + r, k = k0 + threadIdx.x;
    tile[r][threadIdx.x] = (u < N && k < K) ? src[(size_t)iperm[u] * Kp + k] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, u = u0 + threadIdx.x;
    if (k < K && u < N) dst[(size_t)k * N + u] = tile[threadIdx.x][r];
  }
}

// Initial state of every (bus, case) element.  va_t / vm_t / vms_t are
// case-minor FP64 inputs or NULL (flat start / the grid's set-points).
template <class R> struct InitArgs {
  using C = typename Prec<R>::C;
  using M = typename Prec<R>::M;
  int N, K, Kp;
  int enforce_fixed;         // 1: slack angle and pv/slack |V| set from the specification
  const uint8_t* type;
  const double* vmset_grid;  // [N]
  const double* vms_t;       // [N][Kp] or NULL
  const double* va_t;        // [N][Kp] ([N] if shared_start) or NULL
  const double* vm_t;
  int shared_start;          // 1: va_t / vm_t hold one state [N] for every case
  double va_slack;
  const double* p64;         // per-case spec (FP64, [N][Kp]) or NULL
  const double* q64;
  R* p;                      // per-case working-precision copies
  R* q;
  typename Prec<R>::MS* ms;
  C* V;
  Mom<R>* os;
};

template <class R>
__global__ void k_init(InitArgs<R> a) {
  using M = typename Prec<R>::M;
  const size_t n = (size_t)a.N * a.Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.Kp), k = (int)(e % a.Kp);
    const int ty = a.type[i];
    double th = 0.0, vm = 1.0;
    if (k < a.K) {
      if (a.va_t) {
        const size_t si = a.shared_start ? (size_t)i : e;
        th = a.va_t[si];
        vm = a.vm_t[si];
      }
      if (a.enforce_fixed || !a.va_t) {
        const double set = a.vms_t ? a.vms_t[e] : a.vmset_grid[i];
        if (ty != BUS_PQ) vm = set;
        if (ty == BUS_SLACK) th = a.va_slack;
      }
    }
    const M mth = mfrom<M>(th), mvm = mfrom<M>(vm);
    a.ms[e] = ms_make(mth, mvm);
    a.V[e] = volt(mth, mvm);
    a.os[e] = Mom<R>{R(0), R(0), R(0), R(0)};
    if (a.p64) {
      a.p[e] = (R)a.p64[e];
      a.q[e] = (R)a.q64[e];
    }
  }
}

// Per-case scalar state and N-1 corrections.  outage (user branch index or
// -1) may be NULL.  Branch data are FP64 in internal bus order.
template <class R> struct CaseInitArgs {
  using C = typename Prec<R>::C;
  int K, Kp;
  const int32_t* outage;
  const int32_t* br_f;
  const int32_t* br_t;
  const double* br_r;
  const double* br_x;
  const double* br_bch;
  const double* br_tap;
  int32_t* of;
  int32_t* ot;
  C* yff;
  C* yft;
  C* ytt;
  double2* yff64;
  double2* yft64;
  double2* ytt64;
  int32_t* active;
  int32_t* iters;
  int32_t* status;
  double* lr;
  double* best;
  int32_t* bad;
  int32_t* cool;
  R* step_size;
  R* isbc2;
  double* b1t;
  double* b2t;
  int32_t* cand;
  unsigned int* mx32;
  unsigned long long* maxmis;
  double* loss64;
  double lr0, beta1, beta2;
  int opt;
};

template <class R>
__global__ void k_case_init(CaseInitArgs<R> a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.Kp) return;
  const bool real = k < a.K;
  a.active[k] = real ? 1 : 0;
  a.iters[k] = 0;
  a.status[k] = CASE_MAX_ITER;
  a.lr[k] = a.lr0;
  a.best[k] = __longlong_as_double(0x7ff0000000000000LL);  // +inf
  a.bad[k] = 0;
  a.cool[k] = 0;
  a.step_size[k] = (R)(a.opt == OPT_ADAM ? a.lr0 / (1.0 - a.beta1) : a.lr0);
  a.isbc2[k] = (R)(a.opt == OPT_ADAM ? 1.0 / sqrt(1.0 - a.beta2) : 1.0);
  a.b1t[k] = 1.0;  // beta^0: the forward pass multiplies in beta before each step
  a.b2t[k] = 1.0;
  a.cand[k] = 1;
  a.mx32[k] = 0u;
  a.maxmis[k] = 0ULL;
  a.loss64[k] = 0.0;
  int ell = (real && a.outage) ? a.outage[k] : -1;
  if (ell < 0) {
    a.of[k] = -1;
    a.ot[k] = -1;
    return;
  }
  // pi-model block of the outaged branch (removed from the shared Y_bus)
  const double r = a.br_r[ell], x = a.br_x[ell], bch = a.br_bch[ell];
  const double tau = (a.br_tap[ell] == 0.0) ? 1.0 : a.br_tap[ell];
  const double d = r * r + x * x, gs = r / d, bs = -x / d, t2 = tau * tau;
  const double2 ff = make_double2(gs / t2, (bs + 0.5 * bch) / t2);
  const double2 ft = make_double2(-gs / tau, -bs / tau);
  const double2 tt = make_double2(gs, bs + 0.5 * bch);
  a.of[k] = a.br_f[ell];
  a.ot[k] = a.br_t[ell];
  a.yff64[k] = ff;
  a.yft64[k] = ft;
  a.ytt64[k] = tt;
  a.yff[k] = mkc((R)ff.x, (R)ff.y);
  a.yft[k] = mkc((R)ft.x, (R)ft.y);
  a.ytt[k] = mkc((R)tt.x, (R)tt.y);
}

// master (theta, |V|) -> FP64 (for the solution output)
template <class MS>
__global__ void k_master64(const MS* __restrict__ src, double* __restrict__ th, double* __restrict__ vm, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const MS s = src[e];
    th[e] = mval(ms_th(s));
    vm[e] = mval(ms_vm(s));
  }
}

// working precision -> FP64, optional scale (outputs of the evaluation calls)
template <class R>
__global__ void k_widen(const R* __restrict__ src, double* __restrict__ dst, size_t n, size_t stride, double scale) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = scale * (double)src[e * stride];
}

// Y_bus values from per-branch series admittance (g + jb), charging and taps,
// one thread per internal row: off-diagonal entries -y_s/tau, diagonal the
// sum of the incident branches' end contributions.
struct YValArgs {
  int N;
  const int32_t* rp;
  const int32_t* col;
  const int32_t* ebr;
  const int32_t* br_f;  // internal from-bus
  const double* g;      // [M] user branch order
  const double* b;
  const double* bch;
  const double* itap;   // 1 / tap per branch
  int4* ent32;
  double2* val64;
};

__global__ void k_ybus_values(YValArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  double dr = 0.0, di = 0.0;
  int pd = -1;
  for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
    const int ell = a.ebr[p];
    if (ell < 0) { pd = p; continue; }
    const double it = a.itap[ell], it2 = it * it;
    const double gs = a.g[ell], bs = a.b[ell], sh = 0.5 * a.bch[ell];
    const double vr = -gs * it, vi = -bs * it;
    a.val64[p] = make_double2(vr, vi);
    a.ent32[p] = make_int4(a.col[p], __float_as_int((float)vr), __float_as_int((float)vi), 0);
    if (a.br_f[ell] == i) { dr += gs * it2; di += (bs + sh) * it2; }
    else { dr += gs; di += bs + sh; }
  }
  if (pd >= 0) {
    a.val64[pd] = make_double2(dr, di);
    a.ent32[pd] = make_int4(i, __float_as_int((float)dr), __float_as_int((float)di), 0);
  }
}

// Branch-parameter gradients, summed over cases (one thread per
// (branch, case)): with H_ik = w_i V_k (w = c conj V),
//   E = H_ff/tau^2 + H_tt - (H_ft + H_tf)/tau,
//   dL/dg = Re E, dL/db = -Im E, dL/db_ch = -Im(H_ff/tau^2 + H_tt)/2.
template <class R> struct EdgeArgs {
  using C = typename Prec<R>::C;
  int M, K, Kp, lanes;
  const int32_t* br_f;
  const int32_t* br_t;
  const double* itap;  // 1 / tap per branch
  const C* V;
  const C* W;
  double* d_g;
  double* d_b;
  double* d_bch;
};

template <class R>
__global__ void __launch_bounds__(1024) k_edge_grad(EdgeArgs<R> a) {
  using C = typename Prec<R>::C;
  const Map mp = thread_map(a.lanes);
  const int k = mp.k;
  for (int ell0 = mp.row0 - mp.rsub; ell0 < a.M; ell0 += mp.rstride) {
    const int ell = ell0 + mp.rsub;
    R eg = 0, eb = 0, ec = 0;
    if (ell < a.M && k < a.K) {
      const int f = a.br_f[ell], t = a.br_t[ell];
      const R it = (R)a.itap[ell], it2 = it * it;
      const size_t Kp = (size_t)a.Kp;
      const C wf = a.W[(size_t)f * Kp + k], wt = a.W[(size_t)t * Kp + k];
      const C vf = a.V[(size_t)f * Kp + k], vt = a.V[(size_t)t * Kp + k];
      const C hff = mkc(wf.x * vf.x - wf.y * vf.y, wf.x * vf.y + wf.y * vf.x);
      const C htt = mkc(wt.x * vt.x - wt.y * vt.y, wt.x * vt.y + wt.y * vt.x);
      const C hft = mkc(wf.x * vt.x - wf.y * vt.y, wf.x * vt.y + wf.y * vt.x);
      const C htf = mkc(wt.x * vf.x - wt.y * vf.y, wt.x * vf.y + wt.y * vf.x);
      const R er = hff.x * it2 + htt.x - (hft.x + htf.x) * it;
      const R ei = hff.y * it2 + htt.y - (hft.y + htf.y) * it;
      eg = er;
      eb = -ei;
      ec = -(hff.y * it2 + htt.y) * R(0.5);
    }
    for (int off = 1; off < a.lanes; off <<= 1) {
      eg += __shfl_xor_sync(0xffffffffu, eg, off);
      eb += __shfl_xor_sync(0xffffffffu, eb, off);
      ec += __shfl_xor_sync(0xffffffffu, ec, off);
    }
    if (mp.kl == 0 && ell < a.M) {
      if (a.d_g) atomicAdd(a.d_g + ell, (double)eg);
      if (a.d_b) atomicAdd(a.d_b + ell, (double)eb);
      if (a.d_bch) atomicAdd(a.d_bch + ell, (double)ec);
    }
  }
}

}  // namespace dpf
