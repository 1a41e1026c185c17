// Internal definitions shared by the host-only and the CUDA parts of libdpf.
#pragma once

#include <nvtx3/nvToolsExt.h>  // header-only NVTX (ranges are no-ops without an attached tool)
#include <stdint.h>
#include <vector_types.h>  // int4, double2 (CUDA headers; no CUDA calls here)

#include <string>
#include <vector>

#include "dpf.h"

namespace dpf {

// A named NVTX range over a scope: the phases of the library's calls appear
// on Nsight timelines (and can filter ncu captures with --nvtx-include).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Record a failure for dpf_last_error() and return `code`.
int fail(int code, const char* fmt, ...);
void clear_error();

// Device copy of Y_bus and of the grid data, in the internal bus order.
struct DeviceYbus {
  bool ready = false;
  int device = -1;
  int4* ent32 = nullptr;        // [nnz] {col, re bits, im bits, 0}: one 16-byte load per nonzero
  int32_t* row_ptr = nullptr;   // [n+1]
  int32_t* prow_ptr = nullptr;  // [n+1] rows padded to multiples of 4 entries
  int32_t* ppos = nullptr;      // [prow_ptr[n]] CSR position of a padded slot, -(row+1) for a pad
  int32_t* col = nullptr;       // [nnz]
  double2* val64 = nullptr;     // [nnz]
  float2* dcval = nullptr;      // [nnz] DC matrix B (susceptances 1/(x tau)) in the same CSR, as
                                //   double-float pairs (hi, lo): hi + lo is the FP64 value
  float2* dcinv = nullptr;      // [n] 1 / B_ii (0 where B_ii = 0), the Jacobi preconditioner, ditto
  int32_t* ebr = nullptr;       // [nnz] branch of an off-diagonal entry, -1 on the diagonal
  int32_t* dpos = nullptr;      // [n] position of the diagonal entry in its row
  uint8_t* type = nullptr;      // [n]
  double* p64 = nullptr;        // [n] grid injections (internal order)
  double* q64 = nullptr;
  double* vmset = nullptr;      // [n]
  float* p32 = nullptr;
  float* q32 = nullptr;
  int32_t* perm = nullptr;      // [n] internal -> user bus index
  int32_t* iperm = nullptr;     // [n] user -> internal bus index
  int32_t* br_f = nullptr;      // [m] internal bus index of the from-bus
  int32_t* br_t = nullptr;
  double* br_r = nullptr;       // [m]
  double* br_x = nullptr;
  double* br_bch = nullptr;
  double* br_tap = nullptr;
  double* br_itap = nullptr;    // [m] 1 / tap (tap 0 read as 1): no division on the device
  uint8_t* bridge = nullptr;    // [m]
};

}  // namespace dpf

struct dpf_ybus {
  int32_t n = 0, m = 0, nnz = 0;
  int32_t n_pv = 0, n_pq = 0, m_loss = 0;   // m_loss = |pv| + 2|pq|
  int32_t slack = -1;                        // user index
  double va_slack = 0.0;
  // user-order CSR (FP64) and grid data
  std::vector<int32_t> row_ptr, col, dpos, ebr;
  std::vector<double> val_re, val_im;
  std::vector<uint8_t> bus_type;
  std::vector<double> p_spec, q_spec, vm_set;
  std::vector<int32_t> f_bus, t_bus;
  std::vector<double> r, x, b_ch, tap;
  std::vector<uint8_t> bridge;
  // internal order: perm[new] = old, iperm[old] = new; CSR in the new order
  std::vector<int32_t> perm, iperm;
  std::vector<int32_t> irow_ptr, icol, idpos, iebr;
  std::vector<int32_t> iprow_ptr, ippos;     // padded rows (see DeviceYbus)
  std::vector<double> ival_re, ival_im;
  dpf::DeviceYbus dev;
};

namespace dpf {
// Per-branch pi-model blocks (y_ff, y_ft, y_tt; y_tf == y_ft), FP64.
void branch_block(double r, double x, double b_ch, double tap, double out[6]);
}  // namespace dpf
