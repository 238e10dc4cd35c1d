// Host side of the C ABI declared in include/fgfrft.h: argument checks, plan
// layout, the offline driver (Algorithm 1, offline part) and the dispatch of the
// online calls (Def. 1, Def. 2, Props. 2-3) onto the kernels.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc.h"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Layout {
  int64_t blk_elems, Np, plane_elems, Kp, planeT, hplane;
  int nt;
  size_t off_c64, off_f16, off_f16T, off_h16, total;
};

Layout plan_layout(int64_t N, int L_max, int storage) {
  Layout l{};
  const int nblk = 2 * L_max + 2;
  l.blk_elems = round_up(N * N, 32);
  l.Np = round_up(N, 8);
  l.plane_elems = round_up(N * l.Np, 128);
  size_t off = kAlign;  // status word area
  l.off_c64 = off;
  if (storage & FGFRFT_STORE_C64) off = align_up(off + (size_t)nblk * l.blk_elems * sizeof(float2));
  l.off_f16 = off;
  if (storage & FGFRFT_STORE_SPLIT_F16) off = align_up(off + (size_t)nblk * 4 * l.plane_elems * sizeof(__half));
  l.Kp = round_up(nblk, 8);
  l.planeT = round_up(N * N, 128);  // entries per chunk plane of the entry-major copy
  l.off_f16T = off;
  if (storage & FGFRFT_STORE_ENTRY_F16) off = align_up(off + (size_t)4 * l.Kp * l.planeT * sizeof(__half));
  l.nt = (int)((N + 63) / 64);
  l.hplane = (int64_t)l.nt * l.nt * 4096;
  l.off_h16 = off;
  if (storage & FGFRFT_STORE_HALF) off = align_up(off + (size_t)(L_max + 2) * 2 * l.hplane * sizeof(float));
  l.total = off;
  return l;
}

inline bool aligned(const void* p, size_t a = kAlign) { return ((uintptr_t)p % a) == 0; }

#define CK(expr)                                   \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return FGFRFT_ERR_CUDA; \
  } while (0)

// x (finite) is an integer: every double of magnitude >= 2^52 is; below, the truncation
// to int64 is exact and compares equal only for integers.
inline bool is_integer(double x) { return fabs(x) >= 4503599627370496.0 || x == (double)(int64_t)x; }

// Host copy of the orders, validated.  Returns FGFRFT_OK or an error code.  (Runs once per
// call over B orders: B is 16384 on the image-graph batch, so the loop is kept cheap.)
int gather_orders(const double* alpha_host, int64_t B, int L, int flags, std::vector<double>& out) {
  if (!alpha_host || B < 1) return FGFRFT_ERR_INVALID_ARG;
  out.resize((size_t)B);
  const bool shared = (flags & FGFRFT_SHARED_ALPHA) != 0;
  const double Ld = (double)L;
  for (int64_t j = 0; j < B; ++j) {
    const double a = shared ? alpha_host[0] : alpha_host[j];
    if (!isfinite(a)) return FGFRFT_ERR_INVALID_ARG;
    if (fabs(a) > Ld && is_integer(a)) return FGFRFT_ERR_UNSUPPORTED;
    out[(size_t)j] = a;
  }
  return FGFRFT_OK;
}

// Runs of equal orders: (start, length).
using Runs = std::vector<std::pair<int64_t, int64_t>>;
Runs order_runs(const std::vector<double>& a) {
  Runs runs;
  int64_t s = 0;
  for (int64_t j = 1; j <= (int64_t)a.size(); ++j) {
    if (j == (int64_t)a.size() || a[(size_t)j] != a[(size_t)s]) {
      runs.push_back({s, j - s});
      s = j;
    }
  }
  return runs;
}

// The small host tables of one call (orders, tile and group tables): read by the kernels
// straight from pinned host memory (fg_stage), or copied into the work buffer when no slot
// is free.  The slots are released, on the call's stream, when the guard goes out of scope,
// after every kernel of the call is enqueued.
struct Staged {
  cudaStream_t s;
  int tok[8];
  int n = 0;
  bool failed = false;
  bool capturing;  // a graph replays later: tables go into the work buffer (fg_upload)
  explicit Staged(cudaStream_t st) : s(st), capturing(fg_capturing(st)) {}
  Staged(const Staged&) = delete;
  Staged& operator=(const Staged&) = delete;
  ~Staged() {
    for (int i = 0; i < n; ++i) fg_stage_done(tok[i], s);
  }
  // device-readable copy of src; fallback: a stream copy to dev_fallback (in the work buffer)
  template <class T>
  const T* put(const T* src, size_t count, T* dev_fallback) {
    const void* dev = nullptr;
    const int t = n < 8 && !capturing ? fg_stage(src, count * sizeof(T), &dev) : -1;
    if (t >= 0) {
      tok[n++] = t;
      return static_cast<const T*>(dev);
    }
    if (fg_h2d(dev_fallback, src, count * sizeof(T), s) != cudaSuccess) failed = true;
    return dev_fallback;
  }
};

// Work forked onto the auxiliary stream (fg_fork) is joined back into the call's stream
// before the call returns, also on an error path, so nothing of the call outlives it off s.
struct AuxJoin {
  cudaStream_t aux;
  cudaStream_t s;
  AuxJoin(const AuxJoin&) = delete;
  AuxJoin& operator=(const AuxJoin&) = delete;
  ~AuxJoin() { join(); }
  cudaError_t join() {
    const cudaError_t e = fg_join(aux, s);
    aux = nullptr;
    return e;
  }
};

// Sequential sub-allocator over a caller work buffer (nullptr base = sizing only).
struct Carve {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off = align_up(off + count * sizeof(T));
    return p;
  }
};

constexpr int kAssembledMinRun = 64;

// Classification of the lambda = -1 eigenvalues (offline projector).
constexpr int kMaxSquarings = 46;           // adaptive route: at most 2^46-th power of S
constexpr double kNeg1TolMin = 1e-5;        // fixed threshold: FP64 resolves 1 - g^2/4 down to here
constexpr double kNeg1TolMax = 0.5;
constexpr double kAmbiguousGap = 1e-6;      // adaptive route: complement eigenvalues closer to -1 are refused
constexpr double kResidualFloor = 1e-10;    // adaptive route: |lambda + 1| of the counted eigenvalues below this
constexpr int kRefineRounds = 3;            // adaptive route: separations of the counted set
constexpr double kGapBracket = 1.01;        // min_gap bracket: upper / lower bound at most this
constexpr int kMaxGapPower = 52;            // ... or the bracket of S^(2^52), whichever comes first

// Squarings that take s = 1 - tol^2/4 to at most 1/2: 2^m >= 4 ln 2 / tol^2.
int squarings_for_tol(double tol) {
  const double x = 4.0 * 0.6931471805599453 / (tol * tol);
  int m = 0;
  while (ldexp(1.0, m) < x && m < 60) ++m;
  return std::max(m, 1);
}

int choose_path(const fgfrft_plan_s* p, const Runs& runs, int flags) {
  int path = flags & FGFRFT_PATH_MASK;
  if (path) return path;
  if (flags & FGFRFT_REAL_OUTPUT) return FGFRFT_PATH_ASSEMBLED;  // real outputs come from assembled Q
  const bool tensor = (p->storage & FGFRFT_STORE_SPLIT_F16) != 0 && fg_tc_available();
  if (!p->f16 && !p->c64)  // half stack only: assemble per order group, then Q X
    return fg_tc_available() ? FGFRFT_PATH_ASSEMBLED : FGFRFT_PATH_PLAIN;
  int64_t min_run = INT64_MAX;
  for (auto& r : runs) min_run = std::min(min_run, r.second);
  if (min_run >= kAssembledMinRun) {
    if (tensor) return FGFRFT_PATH_ASSEMBLED;
    return (p->storage & FGFRFT_STORE_C64) ? FGFRFT_PATH_PLAIN : FGFRFT_PATH_STACKED_FP32;
  }
  return tensor ? FGFRFT_PATH_STACKED : FGFRFT_PATH_STACKED_FP32;
}

// Path of fgfrft_grad: long runs of one order assemble Q and dQ/dalpha per run (assembled
// path on the tensor cores, else the plain path); short runs use the stacked form.  A plan
// with the half stack only always assembles.
int grad_path(const fgfrft_plan_s* p, const Runs& runs, int flags) {
  int path = flags & FGFRFT_PATH_MASK;
  if (path) return path;
  const bool tc = fg_tc_available();
  const bool single = p->h32 || p->c64 || (p->real && p->f16);  // single-order kernels available
  if (!p->f16 && !p->c64) return tc ? FGFRFT_PATH_ASSEMBLED : FGFRFT_PATH_PLAIN;
  int64_t min_run = INT64_MAX;
  for (auto& r : runs) min_run = std::min(min_run, r.second);
  if (min_run >= kAssembledMinRun && single) return tc ? FGFRFT_PATH_ASSEMBLED : FGFRFT_PATH_PLAIN;
  return (p->f16 && tc) ? FGFRFT_PATH_STACKED : FGFRFT_PATH_STACKED_FP32;
}

// Work layout of fgfrft_assemble (and of the assembly stage of the assembled path).
struct AssembleWork {
  double* alpha_dev = nullptr;
  float2* coef = nullptr;    // single-order kernels: coefficient tables
  float2* coefd = nullptr;   // derivative coefficients (dual assembly dQ/dalpha)
  __half* Cs = nullptr;      // tensor: split coefficients [4][A][Kp] ([4][128][2 L_max] for the pair assembly)
  int* col_exp = nullptr;
  float* diag = nullptr;     // pair assembly: c_0 of each order
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  bool tensor = false;
  size_t bytes = 0;
};

AssembleWork carve_assemble(const fgfrft_plan_s* p, char* base, int64_t A, int L, bool dual = false) {
  AssembleWork w;
  Carve c{base};
  // one order streams best through the single-order kernels; more orders (or no c64
  // stack) use the tensor-core GEMM over the entry-major stack.  The dual assembly
  // (Q and dQ/dalpha) runs on the single-order kernels.
  w.tensor = !dual && p->f16T != nullptr && (A >= 2 || p->c64 == nullptr) && fg_tc_available();
  w.alpha_dev = c.take<double>((size_t)A);
  if (w.tensor) {
    // the pair assembly takes 128 coefficient rows (64 orders and their mirrors) per launch
    const int64_t rows = p->pair ? std::max<int64_t>(A, 128) : A;
    w.Cs = c.take<__half>((size_t)4 * rows * p->Kp);
    w.col_exp = c.take<int>((size_t)rows);
    if (p->pair) w.diag = c.take<float>((size_t)std::min<int64_t>(A, 64));
    w.scratch_bytes = fg_tc_assemble_scratch_bytes(p->N * p->N, A);
    w.scratch = c.take<char>(w.scratch_bytes);
  } else {
    w.coef = c.take<float2>((size_t)(2 * L + 2) * A);
    if (dual) w.coefd = c.take<float2>((size_t)(2 * L + 2) * A);
  }
  w.bytes = c.off;
  return w;
}

// Enqueue the fused assembly of A orders into Qc (c64 [A][N*N]) or Qs (split planes).
// alpha_host (optional): the same orders on the host.
// *pair_out (optional) is set when Qs holds pair-structured operators (the grouped GEMM then
// reads the left of each row tile's diagonal block from planes 2, 3; see TcGroupedArgs::pair).
cudaError_t run_assemble(const fgfrft_plan_s* p, const AssembleWork& w, const double* alpha_dev, int64_t A, int L,
                         float2* Qc, __half* Qs, cudaStream_t s, const double* alpha_host = nullptr,
                         bool* pair_out = nullptr) {
  const int b0 = blk_of_power(p, -L), nb = 2 * L + 1, pb = blk_of_P(p);
  if (pair_out) *pair_out = false;
  if (w.tensor && p->pair && Qs && !Qc) {
    // one pass over the pair stack per 64 orders: Q_a[i][k] and Q_a[k][i] of every entry pair
    for (int64_t a0 = 0; a0 < A; a0 += 64) {
      const int64_t na = std::min<int64_t>(64, A - a0);
      cudaError_t e = fg_coeff_planes_pair(alpha_dev + a0, na, L, p->L_max, w.Cs, w.col_exp, w.diag, s,
                                           alpha_host ? alpha_host + a0 : nullptr);
      if (e != cudaSuccess) return e;
      TcAssembleArgs ta{};
      ta.pair_stack = p->pairS;
      ta.pair_rows = p->pair_rows;
      ta.K2 = 2 * (int64_t)p->L_max;
      ta.diag = w.diag;
      ta.A = na;
      ta.Cs = w.Cs;
      ta.col_exp = w.col_exp;
      ta.Qs = Qs + a0 * 4 * p->qplane;
      ta.N = p->N;
      ta.Np = p->Np;
      ta.plane_elems = p->qplane;
      ta.scratch = w.scratch;
      ta.scratch_bytes = w.scratch_bytes;
      ta.status = p->dstatus;
      ta.real_a = true;
      ta.skip_im = true;
      ta.re_only = true;
      if ((e = fg_tc_assemble(ta, s)) != cudaSuccess) return e;
    }
    if (pair_out) *pair_out = true;
    return cudaSuccess;
  }
  if (w.tensor) {
    cudaError_t e = fg_coeff_planes(alpha_dev, A, L, p->L_max, p->Kp, w.Cs, w.col_exp, s, alpha_host);
    if (e != cudaSuccess) return e;
    TcAssembleArgs ta{};
    ta.entry_stack = p->f16T;
    ta.entries = p->N * p->N;
    ta.K = p->nblk;
    ta.Kp = p->Kp;
    ta.planeT = p->planeT;
    ta.A = A;
    ta.Cs = w.Cs;
    ta.col_exp = w.col_exp;
    ta.Qc = Qc;
    ta.Qs = Qs;
    ta.N = p->N;
    ta.Np = p->Np;
    ta.plane_elems = p->qplane;
    ta.scratch = w.scratch;
    ta.scratch_bytes = w.scratch_bytes;
    ta.status = p->dstatus;
    ta.real_a = p->real;
    ta.skip_im = p->real && p->r_neg1 == 0 && Qs != nullptr;
    ta.re_only = p->real && p->r_neg1 == 0;  // real blocks, P = 0: every Q_a is real
    return fg_tc_assemble(ta, s);
  }
  if (p->h32) {  // half stack: per order, pairs of transposed tiles (half the bytes)
    cudaError_t e = fg_coeffs(alpha_dev, (int)A, L, false, w.coef, nullptr, 1, 2 * L + 2, s);
    if (e != cudaSuccess) return e;
    for (int64_t a = 0; a < A; ++a) {
      e = fg_assemble_half(p->h32, p->hplane, p->nt, p->L_max, L, !p->real, p->r_neg1 > 0, p->N, p->Np,
                           w.coef + a * (2 * L + 2), Qc ? Qc + a * p->N * p->N : nullptr,
                           Qs ? Qs + a * 4 * p->qplane : nullptr, p->qplane,
                           !(p->real && p->r_neg1 == 0), p->dstatus, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!p->c64 && p->real && p->f16) {  // real split planes only: per order, the two real planes
    cudaError_t e = fg_coeffs(alpha_dev, (int)A, L, false, w.coef, nullptr, 1, 2 * L + 2, s);
    if (e != cudaSuccess) return e;
    for (int64_t a = 0; a < A; ++a) {
      e = fg_assemble_single_real(p->f16, 4 * p->plane_elems, p->plane_elems, b0, nb, pb, p->N, p->Np,
                                  w.coef + a * (2 * L + 2), Qc ? Qc + a * p->N * p->N : nullptr,
                                  Qs ? Qs + a * 4 * p->qplane : nullptr, p->qplane, p->r_neg1 > 0, p->dstatus, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = fg_coeffs(alpha_dev, (int)A, L, false, w.coef, nullptr, A, 1, s);
  if (e != cudaSuccess) return e;
  if (A == 1 && p->real && p->f16)  // one order, real F: stream the two real split planes
    return fg_assemble_single_real(p->f16, 4 * p->plane_elems, p->plane_elems, b0, nb, pb, p->N, p->Np, w.coef, Qc,
                                   Qs, p->qplane, p->r_neg1 > 0, p->dstatus, s);
  if (A == 1)  // one order: the bulk-copy streaming kernel, c64 or split output
    return fg_assemble_single(p->c64, p->blk_elems, b0, nb, pb, p->N * p->N, w.coef, Qc, p->dstatus, s, Qs, p->N,
                              p->Np, p->qplane);
  return fg_assemble_multi(p->c64, p->blk_elems, b0, nb, pb, p->N, (int)A, w.coef, Qc, Qs, p->Np, p->qplane,
                           p->dstatus, s);
}

// One order on the single-order kernels: coef = [2L+2] (powers at L + l, P at 2L + 1).
cudaError_t assemble_one(const fgfrft_plan_s* p, const float2* coef, int L, float2* Qc, __half* Qs, cudaStream_t s) {
  const int b0 = blk_of_power(p, -L), nb = 2 * L + 1, pb = blk_of_P(p);
  if (p->h32)
    return fg_assemble_half(p->h32, p->hplane, p->nt, p->L_max, L, !p->real, p->r_neg1 > 0, p->N, p->Np, coef, Qc, Qs,
                            p->qplane, !(p->real && p->r_neg1 == 0), p->dstatus, s);
  if (p->real && p->f16)
    return fg_assemble_single_real(p->f16, 4 * p->plane_elems, p->plane_elems, b0, nb, pb, p->N, p->Np, coef, Qc, Qs,
                                   p->qplane, p->r_neg1 > 0, p->dstatus, s);
  if (p->c64)
    return fg_assemble_single(p->c64, p->blk_elems, b0, nb, pb, p->N * p->N, coef, Qc, p->dstatus, s, Qs, p->N, p->Np,
                              p->qplane);
  return cudaErrorInvalidValue;
}

// Q_a and dQ_a/dalpha = sum_l c_l'(a) M_l + j pi e^{j pi a} P (Prop. 3) for A orders, each on
// the single-order kernels; split outputs Qs, dQs ([A][4][qplane]).
cudaError_t run_assemble_dual(const fgfrft_plan_s* p, const AssembleWork& w, const double* alpha_dev, int64_t A,
                              int L, __half* Qs, __half* dQs, cudaStream_t s) {
  cudaError_t e = fg_coeffs(alpha_dev, (int)A, L, false, w.coef, w.coefd, 1, 2 * L + 2, s);
  if (e != cudaSuccess) return e;
  for (int64_t a = 0; a < A; ++a) {
    e = assemble_one(p, w.coef + a * (2 * L + 2), L, nullptr, Qs + a * 4 * p->qplane, s);
    if (e != cudaSuccess) return e;
    e = assemble_one(p, w.coefd + a * (2 * L + 2), L, nullptr, dQs + a * 4 * p->qplane, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Work layout of an apply / grad call; base == nullptr computes the size only.
struct ApplyWork {
  double* alpha_dev = nullptr;
  double* group_alpha_dev = nullptr;
  float2* coef = nullptr;
  float2* coefd = nullptr;
  float2* Qc = nullptr;
  __half* Qs = nullptr;
  float2* dQc = nullptr;  // dual: dQ/dalpha per group (plain path)
  __half* dQs = nullptr;  // dual: dQ/dalpha per group (assembled path)
  __half* Xs = nullptr;
  int* col_exp = nullptr;
  int* bimag = nullptr;
  double* partials = nullptr;
  int2* gtab = nullptr;
  float2* ysplit = nullptr;  // stacked path: partial sums of the block splits
  float2* dsplit = nullptr;
  void* tc_scratch = nullptr;
  size_t tc_scratch_bytes = 0;
  int64_t xs_rows = 0;
  AssembleWork asm_work;
  char* asm_base = nullptr;
  size_t bytes = 0;
};

ApplyWork carve_apply(const fgfrft_plan_s* p, char* base, int64_t B, int L, int path, int64_t groups, bool grad,
                      bool dual = false) {
  ApplyWork w;
  Carve c{base};
  const int nb = 2 * L + 2;
  w.alpha_dev = c.take<double>((size_t)B);
  switch (path) {
    case FGFRFT_PATH_PLAIN:
      w.group_alpha_dev = c.take<double>((size_t)groups);
      w.coef = c.take<float2>((size_t)nb * groups);
      w.Qc = c.take<float2>((size_t)groups * p->N * p->N);
      w.gtab = c.take<int2>((size_t)groups);
      if (dual) {
        w.coefd = c.take<float2>((size_t)nb * groups);
        w.dQc = c.take<float2>((size_t)groups * p->N * p->N);
      }
      break;
    case FGFRFT_PATH_STACKED_FP32:
      w.coef = c.take<float2>((size_t)nb * B);
      w.coefd = c.take<float2>((size_t)nb * B);
      break;
    case FGFRFT_PATH_ASSEMBLED: {
      w.group_alpha_dev = c.take<double>((size_t)groups);
      w.asm_work = carve_assemble(p, nullptr, groups, L, dual);
      w.asm_base = c.take<char>(w.asm_work.bytes);
      w.Qs = c.take<__half>((size_t)groups * 4 * p->qplane);
      if (dual) w.dQs = c.take<__half>((size_t)groups * 4 * p->qplane);
      w.xs_rows = fg_tc_signal_rows(B, groups);
      w.Xs = c.take<__half>((size_t)4 * w.xs_rows * p->Np);
      w.col_exp = c.take<int>((size_t)w.xs_rows);
      w.bimag = c.take<int>(1);
      w.tc_scratch_bytes = fg_tc_scratch_bytes(p->N, B, groups, 1);
      w.tc_scratch = c.take<char>(w.tc_scratch_bytes);
      if (base) w.asm_work = carve_assemble(p, w.asm_base, groups, L, dual);
      break;
    }
    case FGFRFT_PATH_STACKED: {
      w.coef = c.take<float2>((size_t)nb * B);
      w.coefd = c.take<float2>((size_t)nb * B);
      // partial sums of the block splits (few tiles: each tile's blocks over several CTAs)
      const int splits = fg_tc_stacked_splits(p->N, B, nb);
      if (splits > 1) {
        w.ysplit = c.take<float2>((size_t)splits * B * p->N);
        if (dual) w.dsplit = c.take<float2>((size_t)splits * B * p->N);
      }
      w.xs_rows = fg_tc_signal_rows(B, 1);
      w.Xs = c.take<__half>((size_t)4 * w.xs_rows * p->Np);
      w.col_exp = c.take<int>((size_t)w.xs_rows);
      w.bimag = c.take<int>(1);
      w.tc_scratch_bytes = fg_tc_scratch_bytes(p->N, B, 1, nb);
      w.tc_scratch = c.take<char>(w.tc_scratch_bytes);
      break;
    }
    default:
      break;
  }
  if (grad) w.partials = c.take<double>((size_t)B * fg_grad_chunks(p->N));
  w.bytes = c.off;
  return w;
}

const char* kStatusNames[] = {
    "FGFRFT_OK",
    "FGFRFT_ERR_INVALID_ARG: invalid argument",
    "FGFRFT_ERR_UNSUPPORTED: unsupported request (integer order beyond L, L > L_max, or storage missing)",
    "FGFRFT_ERR_NOT_UNITARY: F is not unitary to 1e-8",
    "FGFRFT_ERR_AMBIGUOUS_SPECTRUM: an eigenvalue of F is too close to -1 to classify",
    "FGFRFT_ERR_NO_MEMORY: host allocation failed",
    "FGFRFT_ERR_CUDA: a CUDA call failed",
    "FGFRFT_ERR_TIMEOUT: a bounded device wait ran out",
};

}  // namespace

extern "C" {

const char* fgfrft_strerror(int status) {
  if (status < 0 || status > FGFRFT_ERR_TIMEOUT) return "unknown fgfrft status";
  return kStatusNames[status];
}

int fgfrft_version(void) { return 100; }

size_t fgfrft_plan_bytes(int64_t N, int L_max, int storage) {
  if (N < 1 || N > 65536 || L_max < 0 || L_max > 1000) return 0;
  const int known = FGFRFT_STORE_C64 | FGFRFT_STORE_SPLIT_F16 | FGFRFT_STORE_ENTRY_F16 | FGFRFT_STORE_HALF;
  if ((storage & (FGFRFT_STORE_C64 | FGFRFT_STORE_SPLIT_F16 | FGFRFT_STORE_HALF)) == 0) return 0;
  if (storage & ~known) return 0;
  if ((storage & FGFRFT_STORE_ENTRY_F16) && !(storage & FGFRFT_STORE_SPLIT_F16)) return 0;
  return plan_layout(N, L_max, storage).total;
}

size_t fgfrft_precompute_work_bytes(int64_t N) {
  if (N < 1 || N > 65536) return 0;
  return align_up((size_t)4 * N * N * sizeof(double2)) + kAlign;
}

int fgfrft_precompute(const double* F_dev, int64_t N, int L_max, int storage, const double* W_dev, int64_t r_W,
                      double neg1_tol, double* P_dev, void* plan_mem, size_t plan_bytes, void* work,
                      size_t work_bytes, void* stream, fgfrft_plan* out) {
  if (!out) return FGFRFT_ERR_INVALID_ARG;
  *out = nullptr;
  const size_t need = fgfrft_plan_bytes(N, L_max, storage);
  if (need == 0 || !F_dev || !plan_mem || !work || plan_bytes < need) return FGFRFT_ERR_INVALID_ARG;
  if (work_bytes < fgfrft_precompute_work_bytes(N)) return FGFRFT_ERR_INVALID_ARG;
  if (!aligned(plan_mem) || !aligned(work) || !aligned(F_dev, 16)) return FGFRFT_ERR_INVALID_ARG;
  if (W_dev && (r_W < 0 || r_W > N || !aligned(W_dev, 16))) return FGFRFT_ERR_INVALID_ARG;
  if (P_dev && !aligned(P_dev, 16)) return FGFRFT_ERR_INVALID_ARG;
  if (!(neg1_tol == 0.0 || (neg1_tol >= kNeg1TolMin && neg1_tol <= kNeg1TolMax))) return FGFRFT_ERR_INVALID_ARG;
  if (N > 46340) return FGFRFT_ERR_UNSUPPORTED;  // int GEMM indices
  cudaStream_t s = (cudaStream_t)stream;
  const Layout lay = plan_layout(N, L_max, storage);
  fgfrft_plan_s* p = (fgfrft_plan_s*)calloc(1, sizeof(fgfrft_plan_s));
  if (!p) return FGFRFT_ERR_NO_MEMORY;
  p->N = N;
  p->L_max = L_max;
  p->storage = storage;
  p->nblk = 2 * L_max + 2;
  p->blk_elems = lay.blk_elems;
  p->Np = lay.Np;
  p->plane_elems = lay.plane_elems;
  // plane stride of the assembled split operators (work buffers); a 256-byte skew between
  // planes measured no faster with the chunk-major entry copy, so it equals the stack's
  p->qplane = lay.plane_elems;
  p->bytes = need;
  char* pm = (char*)plan_mem;
  p->dstatus = (uint32_t*)pm;
  p->c64 = (storage & FGFRFT_STORE_C64) ? (float2*)(pm + lay.off_c64) : nullptr;
  p->f16 = (storage & FGFRFT_STORE_SPLIT_F16) ? (__half*)(pm + lay.off_f16) : nullptr;
  p->f16T = (storage & FGFRFT_STORE_ENTRY_F16) ? (__half*)(pm + lay.off_f16T) : nullptr;
  p->h32 = (storage & FGFRFT_STORE_HALF) ? (float*)(pm + lay.off_h16) : nullptr;
  p->nt = lay.nt;
  p->hplane = lay.hplane;
  p->Kp = lay.Kp;
  p->planeT = lay.planeT;

  const int n = (int)N;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  double2* Am = (double2*)work;
  double2* Bm = Am + N * N;
  double2* Cm = Bm + N * N;
  double2* Dm = Cm + N * N;
  double* red = (double*)((char*)work + align_up((size_t)4 * N * N * sizeof(double2)));
  double h[3];
  auto fail = [&](int code) {
    free(p);
    return code;
  };
  auto readback = [&](void) -> bool {
    if (cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    return cudaStreamSynchronize(s) == cudaSuccess;
  };

  if (cudaMemsetAsync(plan_mem, 0, kAlign, s) != cudaSuccess) return fail(FGFRFT_ERR_CUDA);
  // (1) unitarity: ||F^H F - I||_F / sqrt(N)
  if (fg_zgemm(true, false, n, n, n, one, (const double2*)F_dev, n, (const double2*)F_dev, n, zero, Am, n, s) ||
      fg_zaxpby_identity(N, zero, nullptr, one, make_double2(-1.0, 0.0), Am, s) ||
      fg_ztrace_fro(N, Am, nullptr, red, s) || !readback())
    return fail(FGFRFT_ERR_CUDA);
  if (!(sqrt(h[1]) / sqrt((double)N) <= 1e-8)) return fail(FGFRFT_ERR_NOT_UNITARY);
  // real F: every power and the projector are real (FP64 products of real matrices keep
  // exact zero imaginary parts), so the tensor-core paths may skip the imaginary planes
  if (fg_zimag_sq(N, (const double2*)F_dev, red, s) || !readback()) return fail(FGFRFT_ERR_CUDA);
  p->real = (h[0] == 0.0) && (!W_dev);
  // real F: every FP64 product below is of real matrices, formed by the real GEMM (the same
  // values in a quarter of the FP64 work)
  const bool rg = p->real;
  auto gemm = [&](bool ta, bool tb, double2 alpha, const double2* A, const double2* B, double2* C) {
    return fg_zgemm(ta, tb, n, n, n, alpha, A, n, B, n, zero, C, n, s, rg);
  };

  // (2) projector P onto the lambda = -1 eigenspace, into Cm.
  //
  // S = T T^H with T = (I - F)/2 has eigenvalues s_k = 1 - |lambda_k + 1|^2 / 4, exactly 1 on
  // the -1 eigenspace.  After m squarings they are s_k^(2^m) ~ exp(-2^m |lambda_k + 1|^2 / 4).
  // separate(H): square the Hermitian H (in Bm) until every eigenvalue lies in one of the two
  // basins of McWeeny's iteration -- tr(H) - ||H||_F^2 = sum h_k (1 - h_k) < 0.05 puts each
  // below 0.053 or above 0.947 -- or, with a fixed count, exactly that many times and then
  // require the same; purify P <- 3P^2 - 2P^3 into Cm and leave H^(2^m) in Dm.
  auto form_S = [&](double2* dst) -> bool {  // dst = S (uses Am)
    return fg_zaxpby_identity(N, make_double2(-0.5, 0.0), (const double2*)F_dev, zero, make_double2(0.5, 0.0), Am,
                              s) == cudaSuccess &&
           gemm(false, true, one, Am, Am, dst) == cudaSuccess;
  };
  // FP64 rounding moves an eigenvalue that is exactly 1 by about u sqrt(N) per squaring, and
  // 2^m squarings compound it: at most max_sq(N) squarings keep that drift below 0.02.
  const int max_sq =
      std::max(1, std::min(kMaxSquarings, (int)floor(log2(0.02 / (1.1102230246251565e-16 * sqrt((double)N))))));
  int sq_used = 0;
  // drop >= 0: a refinement of a counted set of rank drop; the trace of the powers must first
  // fall below drop - 1/2 (some counted eigenvalue has decayed) before separation counts
  auto separate = [&](int fixed, int drop) -> int {
    double2* cur = Bm;
    double2* tmp = Am;
    bool converged = false;
    const int limit = fixed ? fixed : max_sq;
    int m = 1;
    for (; m <= limit; ++m) {
      if (gemm(false, false, one, cur, cur, tmp) || fg_zherm_sym(N, tmp, s)) return FGFRFT_ERR_CUDA;
      std::swap(cur, tmp);
      if (fg_ztrace_fro(N, cur, nullptr, red, s) || !readback()) return FGFRFT_ERR_CUDA;
      if (fixed && m < fixed) continue;
      if (drop >= 0 && h[0] > drop - 0.5) continue;
      if (h[0] - h[1] < 0.05) {
        converged = true;
        break;
      }
    }
    if (!converged) return FGFRFT_ERR_AMBIGUOUS_SPECTRUM;
    sq_used = m;
    if (cudaMemcpyAsync(Dm, cur, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return FGFRFT_ERR_CUDA;
    for (int it = 0; it < 12; ++it) {
      if (gemm(false, false, one, cur, cur, tmp) ||          // P^2
          gemm(false, false, one, tmp, cur, Cm) ||           // P^3
          fg_ztrace_fro(N, tmp, cur, red, s) || !readback())  // ||P^2 - P||
        return FGFRFT_ERR_CUDA;
      if (fg_zmcweeny(N, tmp, Cm, cur, s) || fg_zherm_sym(N, cur, s)) return FGFRFT_ERR_CUDA;
      if (sqrt(h[1]) < 1e-13 * sqrt((double)N)) break;
    }
    if (cudaMemcpyAsync(Cm, cur, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return FGFRFT_ERR_CUDA;
    return FGFRFT_OK;
  };
  // rank of P = round(tr P) (P = 0 when it rounds to 0), and the residual ||F P + P||_F
  // (= sqrt(sum over the counted eigenvalues of |lambda + 1|^2) for the exact projector)
  int rank = 0;
  double residual = 0.0;
  auto rank_and_residual = [&]() -> int {
    if (fg_ztrace_fro(N, Cm, nullptr, red, s) || !readback()) return FGFRFT_ERR_CUDA;
    rank = (int)llround(h[0]);
    if (rank < 0 || fabs(h[0] - rank) > 1e-6) return FGFRFT_ERR_AMBIGUOUS_SPECTRUM;
    if (rank == 0 && cudaMemsetAsync(Cm, 0, (size_t)N * N * sizeof(double2), s) != cudaSuccess)
      return FGFRFT_ERR_CUDA;
    if (gemm(false, false, one, (const double2*)F_dev, Cm, Am) || fg_zaxpby_identity(N, one, Cm, one, zero, Am, s) ||
        fg_ztrace_fro(N, Am, nullptr, red, s) || !readback())
      return FGFRFT_ERR_CUDA;
    residual = sqrt(h[1]);
    return FGFRFT_OK;
  };
  // Bracket of the largest eigenvalue below 1 of H^(2^m0) - P (held in Dm; Bm is scratch), as
  // a bracket of the smallest |lambda + 1| among the eigenvalues it holds: with mu_k the
  // eigenvalues of (H^(2^m0) - P)^(2^j) and x = 2^(m0 + j),
  // (sum mu^2 / sum mu)^(1/x) <= s_max <= (sum mu)^(1/x), s_max = 1 - g^2 / 4; squared
  // (normalised, its scale kept as a logarithm) until upper / lower <= kGapBracket.
  double gap_lo = INFINITY, gap_hi = INFINITY;
  auto bracket = [&](int m0) -> int {
    if (fg_zaxpby_identity(N, make_double2(-1.0, 0.0), Cm, one, zero, Dm, s)) return FGFRFT_ERR_CUDA;
    double2* T = Dm;
    double2* T2 = Bm;
    double lnc = 0.0;
    double glo = 0.0, ghi = 2.0;
    for (int j = 0;; ++j) {
      if (fg_ztrace_fro(N, T, nullptr, red, s) || !readback()) return FGFRFT_ERR_CUDA;
      const double A = h[0], Bq = h[1];
      const double x = ldexp(1.0, m0 + j);
      if (!(A > 1e-300) || !(Bq > 0.0)) {  // the powers vanish: every s_k below the bound
        const double ln_hi = (lnc + log(1e-300)) / x;
        glo = ln_hi < 0.0 ? 2.0 * sqrt(-expm1(ln_hi)) : 0.0;
        ghi = 2.0;
        break;
      }
      const double ln_hi = (lnc + log(A)) / x;            // log of the upper bound of s_max
      const double ln_lo = (lnc + log(Bq) - log(A)) / x;  // log of the lower bound
      glo = ln_hi < 0.0 ? 2.0 * sqrt(-expm1(ln_hi)) : 0.0;
      ghi = ln_lo < 0.0 ? 2.0 * sqrt(-expm1(ln_lo)) : 0.0;
      if ((glo > 0.0 && ghi <= kGapBracket * glo) || m0 + j >= kMaxGapPower) break;
      // T <- T^2 / ||T||_F^2 (trace 1 for a Hermitian T), c <- c^2 ||T||_F^2
      if (gemm(false, false, make_double2(1.0 / Bq, 0.0), T, T, T2) || fg_zherm_sym(N, T2, s)) return FGFRFT_ERR_CUDA;
      std::swap(T, T2);
      lnc = 2.0 * lnc + log(Bq);
    }
    if (glo < gap_lo) {
      gap_lo = glo;
      gap_hi = std::max(glo, ghi);
    }
    return FGFRFT_OK;
  };
  const double u = 1.1102230246251565e-16;
  int squarings = 0;
  int rc = FGFRFT_OK;
  if (W_dev) {
    // the caller's eigenspace: P = W W^H; the complement's gap from S - P
    if (r_W > 0) {
      if (fg_zgemm(false, true, n, n, (int)r_W, one, (const double2*)W_dev, (int)r_W, (const double2*)W_dev,
                   (int)r_W, zero, Cm, n, s))
        return fail(FGFRFT_ERR_CUDA);
    } else if (cudaMemsetAsync(Cm, 0, (size_t)N * N * sizeof(double2), s) != cudaSuccess) {
      return fail(FGFRFT_ERR_CUDA);
    }
    if ((rc = rank_and_residual())) return fail(rc);
    if (rank < N) {
      if (!form_S(Dm)) return fail(FGFRFT_ERR_CUDA);
      if ((rc = bracket(0))) return fail(rc);
    }
    if (rank > 0 && !(residual <= 1e-6 * sqrt((double)rank))) return fail(FGFRFT_ERR_AMBIGUOUS_SPECTRUM);
  } else if (neg1_tol > 0.0) {
    // fixed threshold: the squaring count sets the boundary at neg1_tol (its guard band is the
    // separation test); the complement's gap from S - P
    if (!form_S(Bm)) return fail(FGFRFT_ERR_CUDA);
    if ((rc = separate(squarings_for_tol(neg1_tol), -1))) return fail(rc);
    squarings = sq_used;
    if ((rc = rank_and_residual())) return fail(rc);
    if (rank < N) {
      if (!form_S(Dm)) return fail(FGFRFT_ERR_CUDA);
      if ((rc = bracket(0))) return fail(rc);
    }
    // the counted eigenvalues lie below ~0.3 neg1_tol
    if (rank > 0 && !(residual <= neg1_tol * sqrt((double)rank))) return fail(FGFRFT_ERR_AMBIGUOUS_SPECTRUM);
  } else {
    // adaptive: separate S at its widest gap; while the counted set holds eigenvalues that
    // are not -1 to FP64 accuracy (residual above the rounding level of P, which grows as
    // u N / gap), separate P S P again within it.  The eigenvalues each round removes join
    // the complement, whose gap is bracketed from the round's last power.
    if (!form_S(Bm)) return fail(FGFRFT_ERR_CUDA);
    bool accepted = false;
    for (int round = 0; round < kRefineRounds && !accepted; ++round) {
      const int prev_rank = rank;
      if ((rc = separate(0, round > 0 ? prev_rank : -1))) return fail(rc);
      squarings += sq_used;
      if ((rc = rank_and_residual())) return fail(rc);
      if (round > 0 && rank >= prev_rank) return fail(FGFRFT_ERR_AMBIGUOUS_SPECTRUM);  // no progress
      if (rank < N && (rc = bracket(sq_used))) return fail(rc);
      const double thr = std::min(1e-6, std::max(kResidualFloor, 64.0 * u * (double)N / std::max(gap_lo, 1e-300)));
      accepted = rank == 0 || residual <= thr * sqrt((double)rank);
      if (!accepted) {
        // H = P S P: the counted eigenvalues' s_k, zero elsewhere
        if (!form_S(Bm) || gemm(false, false, one, Cm, Bm, Dm) || gemm(false, false, one, Dm, Cm, Bm) ||
            fg_zherm_sym(N, Bm, s))
          return fail(FGFRFT_ERR_CUDA);
      }
    }
    if (!accepted) return fail(FGFRFT_ERR_AMBIGUOUS_SPECTRUM);
    if (rank < N && gap_lo < kAmbiguousGap) return fail(FGFRFT_ERR_AMBIGUOUS_SPECTRUM);
  }
  p->r_neg1 = rank;
  p->proj_residual = residual;
  p->squarings = squarings;
  p->min_gap_lo = gap_lo;
  p->min_gap_hi = gap_hi;
  p->neg1_tol = neg1_tol;
  if (P_dev && cudaMemcpyAsync(P_dev, Cm, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(FGFRFT_ERR_CUDA);

  // (3) powers: M_0 = P_c = I - P, M_n = F M_{n-1}; M_{-n} = M_n^H.  Round into storage.
  auto store = [&](int blk, const double2* M, bool conjT) -> bool {
    float2* c = p->c64 ? p->c64 + (int64_t)blk * p->blk_elems : nullptr;
    __half* f = p->f16 ? p->f16 + (int64_t)blk * 4 * p->plane_elems : nullptr;
    if (!c && !f) return true;
    return fg_store_block(N, M, conjT, c, f, p->Np, p->plane_elems, s) == cudaSuccess;
  };
  // half stack: M_0 .. M_L_max at blocks 0 .. L_max, P at L_max + 1
  auto store_half = [&](int hb, const double2* M) -> bool {
    if (!p->h32) return true;
    return fg_store_half(N, M, p->h32 + (int64_t)hb * 2 * p->hplane, p->nt, p->hplane, s) == cudaSuccess;
  };
  if (!store(blk_of_P(p), Cm, false) || !store_half(L_max + 1, Cm)) return fail(FGFRFT_ERR_CUDA);
  if (fg_zaxpby_identity(N, make_double2(-1.0, 0.0), Cm, zero, one, Am, s)) return fail(FGFRFT_ERR_CUDA);
  if (!store(blk_of_power(p, 0), Am, false) || !store_half(0, Am)) return fail(FGFRFT_ERR_CUDA);
  double2* cur = Am;
  double2* nxt = Bm;
  for (int k = 1; k <= L_max; ++k) {
    if (gemm(false, false, one, (const double2*)F_dev, cur, nxt)) return fail(FGFRFT_ERR_CUDA);
    if (!store(blk_of_power(p, k), nxt, false) || !store(blk_of_power(p, -k), nxt, true) || !store_half(k, nxt))
      return fail(FGFRFT_ERR_CUDA);
    std::swap(cur, nxt);
  }
  if (p->f16T && fg_entry_major(p->f16, p->nblk, N, p->Np, p->plane_elems, p->f16T, p->Kp, p->planeT, s))
    return fail(FGFRFT_ERR_CUDA);
  // a real F without a -1 eigenvalue: M_{-l} = M_l^T and M_0 = I, so one row of the 2 L_max
  // powers l != 0 per entry pair (i, k) gives Q[i][k] and Q[k][i]; the pair stack goes into the
  // imaginary planes of the entry-major copy's full chunks (2 (Kp / 32) planeT 32 entries >=
  // 2 (2 L_max) rows, since 32 (Kp / 32) = 2 L_max for L_max % 16 == 0 and rows <= planeT)
  p->pair = false;
  if (p->f16T && p->real && p->r_neg1 == 0 && N % 128 == 0 && fg_tc_pair_fits(L_max)) {
    const int64_t rows = 128 * pair_tiles((int)(N / 128));
    const int64_t nfull = p->Kp / 32;
    if (2 * (int64_t)L_max * rows <= 32 * nfull * p->planeT) {
      p->pairS = p->f16T + 2 * nfull * p->planeT * 32;
      p->pair_rows = rows;
      if (fg_pair_stack(p->f16, L_max, N, p->Np, p->plane_elems, p->pairS, rows, s)) return fail(FGFRFT_ERR_CUDA);
      p->pair = true;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FGFRFT_ERR_CUDA);
  *out = p;
  return FGFRFT_OK;
}

int fgfrft_plan_info(fgfrft_plan p, int64_t* N, int* L_max, int* storage, int* r_neg1, double* proj_residual,
                     int* squarings, size_t* plan_bytes, double* min_gap) {
  if (!p) return FGFRFT_ERR_INVALID_ARG;
  if (N) *N = p->N;
  if (L_max) *L_max = p->L_max;
  if (storage) *storage = p->storage;
  if (r_neg1) *r_neg1 = p->r_neg1;
  if (proj_residual) *proj_residual = p->proj_residual;
  if (squarings) *squarings = p->squarings;
  if (plan_bytes) *plan_bytes = p->bytes;
  if (min_gap) {
    min_gap[0] = p->min_gap_lo;
    min_gap[1] = p->min_gap_hi;
  }
  return FGFRFT_OK;
}

const void* fgfrft_plan_block(fgfrft_plan p, int storage, int l, int64_t* block_stride_elems) {
  if (!p || l < -p->L_max || l > p->L_max + 1) return nullptr;
  const int blk = l == p->L_max + 1 ? blk_of_P(p) : blk_of_power(p, l);
  if (storage == FGFRFT_STORE_C64 && p->c64) {
    if (block_stride_elems) *block_stride_elems = p->blk_elems;
    return p->c64 + (int64_t)blk * p->blk_elems;
  }
  if (storage == FGFRFT_STORE_SPLIT_F16 && p->f16) {
    if (block_stride_elems) *block_stride_elems = 4 * p->plane_elems;
    return p->f16 + (int64_t)blk * 4 * p->plane_elems;
  }
  if (storage == FGFRFT_STORE_HALF && p->h32 && l >= 0) {
    if (block_stride_elems) *block_stride_elems = 2 * p->hplane;
    return p->h32 + (int64_t)l * 2 * p->hplane;  // l = L_max + 1 is P
  }
  return nullptr;
}

int fgfrft_plan_status(fgfrft_plan p, void* stream) {
  if (!p) return FGFRFT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t w = 0;
  CK(cudaMemcpyAsync(&w, p->dstatus, sizeof(w), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (w) {
    CK(cudaMemsetAsync(p->dstatus, 0, sizeof(w), s));
    CK(cudaStreamSynchronize(s));
  }
  if (w & FG_STATUS_WAIT_TIMEOUT) return FGFRFT_ERR_TIMEOUT;
  if (w & FG_STATUS_LAUNCH_MISMATCH) return FGFRFT_ERR_CUDA;
  return FGFRFT_OK;
}

int fgfrft_plan_real(fgfrft_plan p) {
  if (!p) return -FGFRFT_ERR_INVALID_ARG;
  return p->real ? 1 : 0;
}

int fgfrft_plan_pair(fgfrft_plan p) {
  if (!p) return -FGFRFT_ERR_INVALID_ARG;
  return p->pair ? 1 : 0;
}

int fgfrft_plan_destroy(fgfrft_plan p) {
  if (!p) return FGFRFT_ERR_INVALID_ARG;
  free(p);
  return FGFRFT_OK;
}

size_t fgfrft_work_bytes(fgfrft_plan p, int op, const double* alpha_host, int64_t count, int L, int flags) {
  if (!p || count < 1 || L < 0 || L > p->L_max) return 0;
  std::vector<double> a;
  if (op == FGFRFT_OP_ASSEMBLE) {
    if (!alpha_host) return 0;
    return carve_assemble(p, nullptr, count, L).bytes;
  }
  if (gather_orders(alpha_host, count, L, flags, a) != FGFRFT_OK) return 0;
  if (flags & FGFRFT_ADJOINT)
    for (auto& v : a) v = -v;
  const Runs runs = order_runs(a);
  const int path = op == FGFRFT_OP_GRAD ? grad_path(p, runs, flags) : choose_path(p, runs, flags);
  const int64_t groups = (int64_t)runs.size();
  if (op == FGFRFT_OP_GRAD) {
    // the dual forward, the backward at -alpha (the same runs) and the gradient partials
    return carve_apply(p, nullptr, count, L, path, groups, true, true).bytes;
  }
  return carve_apply(p, nullptr, count, L, path, groups, false).bytes;
}

int fgfrft_assemble(fgfrft_plan p, const double* alpha_host, int64_t A, int L, void* Q_dev, void* work,
                    size_t work_bytes, void* stream) {
  if (!p || !alpha_host || A < 1 || !Q_dev || !work || L < 0) return FGFRFT_ERR_INVALID_ARG;
  if (L > p->L_max) return FGFRFT_ERR_UNSUPPORTED;
  if (A > 65535) return FGFRFT_ERR_INVALID_ARG;
  std::vector<double> a;
  int rc = gather_orders(alpha_host, A, L, 0, a);
  if (rc) return rc;
  if (work_bytes < fgfrft_work_bytes(p, FGFRFT_OP_ASSEMBLE, alpha_host, A, L, 0) || !aligned(work) ||
      !aligned(Q_dev, 16))
    return FGFRFT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  AssembleWork w = carve_assemble(p, (char*)work, A, L);
  if (!w.tensor && !p->c64 && !p->h32 && !(p->real && p->f16)) return FGFRFT_ERR_UNSUPPORTED;
  Staged st(s);
  const double* ad = st.put(a.data(), (size_t)A, w.alpha_dev);
  if (st.failed) return FGFRFT_ERR_CUDA;
  CK(run_assemble(p, w, ad, A, L, (float2*)Q_dev, nullptr, s, a.data()));
  return FGFRFT_OK;
}

// runs: order_runs(a) (the caller's; negating every order keeps the runs).
static int apply_impl(fgfrft_plan p, std::vector<double>& a, const Runs& runs, int64_t B, int L, const void* X_dev,
                      void* Y_dev, void* D_dev, int path, void* work, size_t work_bytes, cudaStream_t s,
                      int real_io = 0) {
  const bool x_real = (real_io & FGFRFT_REAL_SIGNALS) != 0, y_real = (real_io & FGFRFT_REAL_OUTPUT) != 0;
  if ((x_real && path != FGFRFT_PATH_ASSEMBLED && path != FGFRFT_PATH_STACKED) ||
      (y_real && (!x_real || path != FGFRFT_PATH_ASSEMBLED || !p->real || p->r_neg1 != 0 || D_dev)))
    return FGFRFT_ERR_UNSUPPORTED;
  const int64_t groups = (int64_t)runs.size();
  ApplyWork w = carve_apply(p, (char*)work, B, L, path, groups, false, D_dev != nullptr);
  if (work_bytes < w.bytes) return FGFRFT_ERR_INVALID_ARG;
  const int n = (int)p->N;
  const int b0 = blk_of_power(p, -L), nb = 2 * L + 1, pb = blk_of_P(p);
  const float2* X = (const float2*)X_dev;
  float2* Y = (float2*)Y_dev;
  Staged st(s);  // the call's host tables; released after the last launch below
  switch (path) {
    case FGFRFT_PATH_PLAIN: {
      if (!p->c64 && !(p->real && p->f16) && !p->h32) return FGFRFT_ERR_UNSUPPORTED;
      if (groups > 65535) return FGFRFT_ERR_UNSUPPORTED;
      std::vector<double> ga((size_t)groups);
      for (int64_t g = 0; g < groups; ++g) ga[(size_t)g] = a[(size_t)runs[(size_t)g].first];
      const double* gad = st.put(ga.data(), ga.size(), w.group_alpha_dev);
      if (st.failed) return FGFRFT_ERR_CUDA;
      // coefficient vectors one per order, contiguous: [groups][2L+2] (and c_l' for the dual)
      CK(fg_coeffs(gad, (int)groups, L, false, w.coef, D_dev ? w.coefd : nullptr, 1, nb + 1, s));
      // per order: stream the stack once into Q_g (one single-order assembly launch each;
      // real F streams the two real split planes), then all Q_g X_g on FP32 CUDA cores in
      // one batched launch
      std::vector<int2> gt((size_t)groups);
      int maxc = 0;
      for (int64_t g = 0; g < groups; ++g) {
        CK(assemble_one(p, w.coef + g * (nb + 1), L, w.Qc + g * p->N * p->N, nullptr, s));
        if (D_dev) CK(assemble_one(p, w.coefd + g * (nb + 1), L, w.dQc + g * p->N * p->N, nullptr, s));
        gt[(size_t)g] = make_int2((int)runs[(size_t)g].first, (int)runs[(size_t)g].second);
        maxc = std::max(maxc, (int)runs[(size_t)g].second);
      }
      const int2* gtd = st.put(gt.data(), gt.size(), w.gtab);
      if (st.failed) return FGFRFT_ERR_CUDA;
      SimtStackArgs sa{};
      sa.A = w.Qc;
      sa.lda = n;
      sa.b0 = 0;
      sa.nb_pow = 1;
      sa.p_blk = -1;
      sa.N = n;
      sa.ncols = (int)B;
      sa.X = X;
      sa.Y = Y;
      sa.groups = gtd;
      sa.group_stride = p->N * p->N;
      sa.max_group_cols = maxc;
      sa.ngroups = (int)groups;
      if (Y) CK(fg_simt_stacked(sa, s));
      if (D_dev) {  // D = (dQ/dalpha) X
        sa.A = w.dQc;
        sa.Y = (float2*)D_dev;
        CK(fg_simt_stacked(sa, s));
      }
      return FGFRFT_OK;
    }
    case FGFRFT_PATH_STACKED_FP32: {
      if (!p->c64) return FGFRFT_ERR_UNSUPPORTED;
      const double* ad = st.put(a.data(), (size_t)B, w.alpha_dev);
      if (st.failed) return FGFRFT_ERR_CUDA;
      CK(fg_coeffs(ad, (int)B, L, false, w.coef, D_dev ? w.coefd : nullptr, B, 1, s));
      SimtStackArgs sa{};
      sa.A = p->c64;
      sa.blk_elems = p->blk_elems;
      sa.lda = n;
      sa.b0 = b0;
      sa.nb_pow = nb;
      sa.p_blk = pb;
      sa.N = n;
      sa.X = X;
      sa.ldcoef = (int)B;
      for (int64_t j0 = 0; j0 < B; j0 += 65535LL * 64) {
        const int64_t nc = std::min<int64_t>(B - j0, 65535LL * 64);
        sa.ncols = (int)nc;
        sa.X = X + j0 * p->N;
        sa.Y = Y ? Y + j0 * p->N : nullptr;
        sa.D = D_dev ? (float2*)D_dev + j0 * p->N : nullptr;
        sa.coef = w.coef + j0;
        sa.coefd = w.coefd + j0;
        CK(fg_simt_stacked(sa, s));
      }
      return FGFRFT_OK;
    }
    case FGFRFT_PATH_ASSEMBLED: {
      if (!fg_tc_available()) return FGFRFT_ERR_UNSUPPORTED;
      if (D_dev ? !(p->h32 || p->c64 || (p->real && p->f16)) : !(p->h32 || (p->f16 && (p->c64 || p->f16T))))
        return FGFRFT_ERR_UNSUPPORTED;
      std::vector<double> ga((size_t)groups);
      std::vector<int64_t> gstart((size_t)groups), gcount((size_t)groups);
      for (int64_t g = 0; g < groups; ++g) {
        ga[(size_t)g] = a[(size_t)runs[(size_t)g].first];
        gstart[(size_t)g] = runs[(size_t)g].first;
        gcount[(size_t)g] = runs[(size_t)g].second;
      }
      // every host table of the call goes up first, so no copy waits in the middle of the call
      std::vector<int4> tiles;
      fg_tc_grouped_tiles(p->N, groups, gstart.data(), gcount.data(),
                          fg_tc_grouped_bn(p->real && p->r_neg1 == 0), tiles);
      if (tiles.size() * sizeof(int4) > w.tc_scratch_bytes) return FGFRFT_ERR_INVALID_ARG;
      const double* gad = st.put(ga.data(), ga.size(), w.group_alpha_dev);
      const int4* tiles_dev = st.put(tiles.data(), tiles.size(), (int4*)w.tc_scratch);
      if (st.failed) return FGFRFT_ERR_CUDA;
      // the signal split runs beside the operator assembly on the auxiliary stream (they
      // share no buffer); the GEMM waits for both
      AuxJoin aux{fg_fork(s), s};
      bool pair = false;
      if (aux.aux)
        CK(fg_split_signals(X, B, p->N, p->Np, w.xs_rows, w.Xs, w.col_exp, aux.aux, w.bimag, x_real));
      if (D_dev)
        CK(run_assemble_dual(p, w.asm_work, gad, groups, L, w.Qs, w.dQs, s));
      else
        CK(run_assemble(p, w.asm_work, gad, groups, L, nullptr, w.Qs, s, ga.data(), &pair));
      const bool split_done = aux.aux != nullptr;
      CK(aux.join());
      TcGroupedArgs ta{};
      ta.tiles_dev = tiles_dev;
      ta.ntiles = (int64_t)tiles.size();
      ta.N = p->N;
      ta.Np = p->Np;
      ta.plane_elems = p->qplane;
      ta.Qs = w.Qs;
      ta.groups = groups;
      ta.gstart = gstart.data();
      ta.gcount = gcount.data();
      ta.X = X;
      ta.Y = Y;
      ta.Xs = w.Xs;
      ta.xs_rows = w.xs_rows;
      ta.col_exp = w.col_exp;
      ta.B = B;
      ta.scratch = w.tc_scratch;
      ta.scratch_bytes = w.tc_scratch_bytes;
      ta.status = p->dstatus;
      ta.real_a = p->real && p->r_neg1 == 0;  // Q = R + j sin(pi a) P is real when P = 0
      ta.bimag = w.bimag;
      ta.x_real = x_real;
      ta.y_real = y_real;
      ta.x_split_done = split_done;
      ta.pair = pair;
      if (Y) CK(fg_tc_grouped_apply(ta, s));
      if (D_dev) {  // D = (dQ/dalpha) X on the same split signals
        ta.Qs = w.dQs;
        ta.Y = (float2*)D_dev;
        ta.x_split_done = split_done || Y != nullptr;
        CK(fg_tc_grouped_apply(ta, s));
      }
      return FGFRFT_OK;
    }
    case FGFRFT_PATH_STACKED: {
      if (!p->f16 || !fg_tc_available()) return FGFRFT_ERR_UNSUPPORTED;
      const double* ad = st.put(a.data(), (size_t)B, w.alpha_dev);
      if (st.failed) return FGFRFT_ERR_CUDA;
      CK(fg_coeffs(ad, (int)B, L, false, w.coef, D_dev ? w.coefd : nullptr, B, 1, s));
      TcStackedArgs ta{};
      ta.N = p->N;
      ta.Np = p->Np;
      ta.plane_elems = p->plane_elems;
      ta.stack = p->f16;
      ta.b0 = b0;
      ta.nb_pow = nb;
      ta.p_blk = pb;
      ta.X = X;
      ta.Y = Y;
      ta.D = (float2*)D_dev;
      ta.coef = w.coef;
      ta.coefd = w.coefd;
      ta.B = B;
      ta.Xs = w.Xs;
      ta.xs_rows = w.xs_rows;
      ta.col_exp = w.col_exp;
      ta.scratch = w.tc_scratch;
      ta.scratch_bytes = w.tc_scratch_bytes;
      ta.status = p->dstatus;
      ta.real_a = p->real;
      ta.bimag = w.bimag;
      ta.x_real = x_real;
      ta.Ysplit = w.ysplit;
      ta.Dsplit = w.dsplit;
      CK(fg_tc_stacked_apply(ta, s));
      return FGFRFT_OK;
    }
    default:
      return FGFRFT_ERR_INVALID_ARG;
  }
}

int fgfrft_apply(fgfrft_plan p, const double* alpha_host, int64_t B, int L, const void* X_dev, void* Y_dev,
                 int flags, void* work, size_t work_bytes, void* stream) {
  if (!p || !alpha_host || B < 1 || !X_dev || !Y_dev || !work || L < 0) return FGFRFT_ERR_INVALID_ARG;
  if (L > p->L_max) return FGFRFT_ERR_UNSUPPORTED;
  const int real_io = flags & (FGFRFT_REAL_SIGNALS | FGFRFT_REAL_OUTPUT);
  if (!aligned(work) || !aligned(X_dev, (real_io & FGFRFT_REAL_SIGNALS) ? 4 : 8) ||
      !aligned(Y_dev, (real_io & FGFRFT_REAL_OUTPUT) ? 4 : 8))
    return FGFRFT_ERR_INVALID_ARG;
  std::vector<double> a;
  int rc = gather_orders(alpha_host, B, L, flags, a);
  if (rc) return rc;
  if (flags & FGFRFT_ADJOINT)
    for (auto& v : a) v = -v;
  const Runs runs = order_runs(a);
  const int path = choose_path(p, runs, flags);
  if (path == FGFRFT_PATH_PLAIN && !p->c64 && !(p->real && p->f16) && !p->h32) return FGFRFT_ERR_UNSUPPORTED;
  return apply_impl(p, a, runs, B, L, X_dev, Y_dev, nullptr, path, work, work_bytes, (cudaStream_t)stream, real_io);
}

int fgfrft_grad(fgfrft_plan p, const double* alpha_host, int64_t B, int L, const void* X_dev, void* Y_dev,
                void* dY_dev, const void* G_dev, void* gradX_dev, float* gradalpha_dev, int flags, void* work,
                size_t work_bytes, void* stream) {
  if (!p || !alpha_host || B < 1 || !work || L < 0) return FGFRFT_ERR_INVALID_ARG;
  if (L > p->L_max) return FGFRFT_ERR_UNSUPPORTED;
  if (!X_dev && !G_dev) return FGFRFT_ERR_INVALID_ARG;
  if (X_dev && !Y_dev && !dY_dev) return FGFRFT_ERR_INVALID_ARG;
  if (G_dev && !gradX_dev && !gradalpha_dev) return FGFRFT_ERR_INVALID_ARG;
  if (gradalpha_dev && !dY_dev) return FGFRFT_ERR_INVALID_ARG;
  if (!aligned(work)) return FGFRFT_ERR_INVALID_ARG;
  std::vector<double> a;
  int rc = gather_orders(alpha_host, B, L, flags & ~FGFRFT_ADJOINT, a);
  if (rc) return rc;
  const Runs runs = order_runs(a);
  const int path = grad_path(p, runs, flags);
  const int64_t groups = (int64_t)runs.size();
  ApplyWork w = carve_apply(p, (char*)work, B, L, path, groups, true, true);
  if (work_bytes < w.bytes) return FGFRFT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (X_dev) {
    rc = apply_impl(p, a, runs, B, L, X_dev, Y_dev, dY_dev, path, work, work_bytes, s);
    if (rc) return rc;
  }
  if (G_dev) {
    if (gradalpha_dev)
      CK(fg_grad_alpha((const float2*)G_dev, (const float2*)dY_dev, B, p->N, gradalpha_dev, w.partials, s,
                       (flags & FGFRFT_SHARED_ALPHA) != 0));
    if (gradX_dev) {
      std::vector<double> na(a);
      for (auto& v : na) v = -v;
      rc = apply_impl(p, na, runs, B, L, G_dev, gradX_dev, nullptr, path, work, work_bytes, s);
      if (rc) return rc;
    }
  }
  return FGFRFT_OK;
}

}  // extern "C"
