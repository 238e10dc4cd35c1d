/*
 * fgfrft.h -- C ABI of libfgfrft, the GB300 (sm_103a) online hot path of the
 * fast graph fractional Fourier transform (FGFRFT).
 *
 * Method (paper: "FGFRFT: Fast Graph Fractional Fourier Transform via Exact
 * Spectral Splitting and Fourier-Series Approximation"):
 *
 *   F        unitary N x N graph Fourier matrix (Sec. III-A), eigenphases
 *            theta_k in (-pi, pi].
 *   P        orthogonal projector onto the lambda = -1 eigenspace, P_c = I - P
 *            (Sec. III-B).
 *   M_l      = F^l P_c for l = -L..L, the cached integer powers (Algorithm 1,
 *            offline part; M_{-l} = M_l^H by Prop. 2 / Eq. "eqefficient_computation").
 *   c_l(a)   = sin(pi (a - l)) / (pi (a - l)) (Sec. III-A).
 *   Q_L^a    = e^{j pi a} P + sum_{l=-L}^{L} c_l(a) M_l        (Def. 1)
 *   Y        = Q_L^a X, one order per signal column              (Def. 2)
 *   dY/da    = j pi e^{j pi a} P X + sum_l c_l'(a) M_l X          (Prop. 3)
 *   Q^H G    = Q_L^{-a} G                                         (Prop. 2)
 *
 * Conventions shared by every call:
 *   - Matrices are row-major.  "c64" means interleaved complex float32
 *     (re, im) pairs, "c128" interleaved complex float64.
 *   - Signals are stored one per row: X[j * N + i] is entry i of signal j
 *     (column j of the N x B matrix X).  Y, dY/da, G and gradX use the same
 *     layout.
 *   - Every pointer named *_dev is device memory owned by the caller; *_host
 *     is host memory read before the call returns.  The library allocates no
 *     device memory: the plan lives in caller memory of fgfrft_plan_bytes()
 *     bytes, scratch in a caller buffer of fgfrft_work_bytes() bytes.
 *   - Device memory passed to one call must not overlap between inputs and
 *     outputs.  A work buffer may be reused by the next call on the same
 *     stream, not by concurrent calls.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without synchronising,
 *     except fgfrft_precompute (which reads reductions back) and
 *     fgfrft_plan_status.
 *   - fgfrft_assemble, fgfrft_apply and fgfrft_grad may be captured into a
 *     CUDA graph (stream capture): the call's orders and host tables are then
 *     carried by the captured kernels and written into the work buffer at
 *     every replay, which reads the signals and writes the outputs at replay
 *     time.  The work buffer of a graph must not be in use by another call
 *     while the graph replays.  (The library's auxiliary stream, on which the
 *     assembled path runs its signal split beside the operator assembly, is
 *     created by the first uncaptured call; a capture before any such call
 *     runs the split in line.)
 *   - Argument errors are detected on the host before anything is enqueued.
 *     CUDA launch errors return FGFRFT_ERR_CUDA.  Errors found by kernels
 *     (a bounded wait that ran out) are recorded in the plan's device status
 *     word and reported by fgfrft_plan_status.
 *   - Orders are host float64.  An order a is an integer iff a == round(a);
 *     then c_l(a) is the Kronecker delta and Q = F^a exactly (Remark 2), which
 *     the stored powers cover only for |a| <= L: larger integer orders return
 *     FGFRFT_ERR_UNSUPPORTED.
 *   - L (0 <= L <= L_max) selects the central blocks -L..L of the stored stack.
 */
#ifndef FGFRFT_H
#define FGFRFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fgfrft_plan_s* fgfrft_plan;

enum fgfrft_status {
  FGFRFT_OK = 0,
  FGFRFT_ERR_INVALID_ARG = 1,        /* bad size, NULL pointer, short buffer, NaN order */
  FGFRFT_ERR_UNSUPPORTED = 2,        /* integer |a| > L, L > L_max, storage missing for a path */
  FGFRFT_ERR_NOT_UNITARY = 3,        /* ||F^H F - I||_F / sqrt(N) above 1e-8 */
  FGFRFT_ERR_AMBIGUOUS_SPECTRUM = 4, /* an eigenvalue too close to -1 to classify in FP64 */
  FGFRFT_ERR_NO_MEMORY = 5,          /* host allocation of the plan record failed */
  FGFRFT_ERR_CUDA = 6,               /* a CUDA call or kernel launch failed */
  FGFRFT_ERR_TIMEOUT = 7,            /* a kernel's bounded wait ran out (status word) */
};

/* Storage of the power stack, a bit set passed to fgfrft_precompute. */
enum fgfrft_storage {
  FGFRFT_STORE_C64 = 1,       /* blocks as c64, 8 B per entry: assembly and FP32 paths */
  FGFRFT_STORE_SPLIT_F16 = 2, /* blocks as four fp16 planes {re_hi, re_lo, im_hi, im_lo}
                                 of the entries scaled by 2^12, 8 B per entry:
                                 tensor-core paths */
  FGFRFT_STORE_ENTRY_F16 = 4, /* an entry-major copy of the split planes: for every entry
                                 of the N x N blocks, the 2 L_max + 2 stored blocks (padded
                                 to Kp, a multiple of 8) in chunks of 32 contiguous values
                                 (chunk-major planes, then a Kp mod 32 tail plane); lets the
                                 fused multi-order assembly run as one tensor-core GEMM.
                                 Requires FGFRFT_STORE_SPLIT_F16. */
  FGFRFT_STORE_HALF = 8,      /* M_0 .. M_{L_max} and P only (L_max + 2 blocks): a negative
                                 power is read as the conjugate transpose of the stored
                                 positive one, M_{-l} = M_l^H (Prop. 2, as Algorithm 1
                                 forms it).  Each block is two FP32 planes (re, im) of
                                 64 x 64 tiles, tiles in row-major order, element (r, c)
                                 of a tile at r * 64 + (c XOR (r mod 32)); 8 B per entry.
                                 Read by the single-order assembly (pairs of transposed
                                 tiles, half the bytes of a full stack), and so by
                                 fgfrft_assemble, the plain and assembled paths of
                                 fgfrft_apply and fgfrft_grad; the stacked paths need
                                 FGFRFT_STORE_SPLIT_F16 or FGFRFT_STORE_C64. */
};

/* Flags of fgfrft_apply / fgfrft_grad. */
enum fgfrft_flags {
  FGFRFT_ADJOINT = 1,             /* apply (Q_L^a)^H = Q_L^{-a} (Prop. 2) */
  FGFRFT_SHARED_ALPHA = 2,        /* alpha_host holds one order used by every column */
  FGFRFT_PATH_PLAIN = 0x10,       /* per order: assemble Q (c64), then FP32 SIMT GEMM */
  FGFRFT_PATH_ASSEMBLED = 0x20,   /* all orders assembled in one pass into split-fp16
                                     operators, then one tensor-core GEMM over groups */
  FGFRFT_PATH_STACKED = 0x40,     /* no assembly: the stacked powers [M_-L..M_L, P] as one
                                     tensor-core GEMM against X, per-column orders */
  FGFRFT_PATH_STACKED_FP32 = 0x80, /* the stacked form on FP32 CUDA cores */
  FGFRFT_REAL_SIGNALS = 0x100,     /* fgfrft_apply: X_dev holds B x N real float32 signals
                                      (imaginary parts zero); tensor-core paths only */
  FGFRFT_REAL_OUTPUT = 0x200       /* fgfrft_apply: Y_dev receives B x N real float32 outputs;
                                      needs FGFRFT_REAL_SIGNALS, a real F without a -1
                                      eigenvalue (then Q is real) and the assembled path */
};
#define FGFRFT_PATH_MASK 0xF0

/* Operation codes of fgfrft_work_bytes. */
enum fgfrft_op { FGFRFT_OP_ASSEMBLE = 1, FGFRFT_OP_APPLY = 2, FGFRFT_OP_GRAD = 3 };

/* Human-readable name of a status code; never NULL. */
const char* fgfrft_strerror(int status);

/* Library version, major * 10000 + minor * 100 + patch. */
int fgfrft_version(void);

/* Bytes of device memory a plan for (N, L_max, storage) occupies: the status
 * word, 2 L_max + 2 blocks of N x N entries (M_{-L_max} .. M_{L_max}, then P)
 * in every full storage requested (L_max + 2 blocks M_0 .. M_{L_max}, P for
 * FGFRFT_STORE_HALF), each storage padded to 256 B.  Returns 0 for invalid
 * arguments (N < 1, L_max < 0, no storage of the blocks, an unknown bit, or
 * FGFRFT_STORE_ENTRY_F16 without FGFRFT_STORE_SPLIT_F16). */
size_t fgfrft_plan_bytes(int64_t N, int L_max, int storage);

/* Bytes of FP64 device scratch fgfrft_precompute needs: 4 N^2 complex128
 * matrices plus a reduction area. */
size_t fgfrft_precompute_work_bytes(int64_t N);

/*
 * Offline part of Algorithm 1, in FP64 on the GPU.
 *   F_dev       N x N complex128 (c128) row-major unitary matrix, device.
 *   L_max       highest stored power (>= 0).
 *   storage     bit set of enum fgfrft_storage.
 *   W_dev       optional N x r complex128 row-major matrix with orthonormal
 *               columns spanning the lambda = -1 eigenspace (Algorithm 1,
 *               "form W"); NULL lets the library find the eigenspace itself:
 *               S = (I - F)(I - F)^H / 4 has eigenvalues s_k = sin^2(theta_k / 2)
 *               = 1 - |lambda_k + 1|^2 / 4, equal to 1 exactly on the lambda = -1
 *               eigenspace; repeated squaring of S followed by McWeeny
 *               purification P <- 3P^2 - 2P^3 gives P (Sec. III-B: I_{-1} = {k :
 *               theta_k = pi}; the paper fixes no tolerance for it).
 *   r_W         number of columns of W_dev (ignored when W_dev is NULL).
 *   neg1_tol    which eigenvalues count as -1 when W_dev is NULL:
 *               0: adaptive, with the oracle's classification (|lambda + 1| <=
 *                  1e-8 is -1) wherever FP64 can certify it.  S is squared until
 *                  its powers separate into the two basins of McWeeny's iteration,
 *                  so the widest gap in |lambda + 1| decides; while the counted set
 *                  holds eigenvalues that are not -1 to FP64 accuracy (its residual
 *                  ||F P + P|| / sqrt(r_neg1) above max(1e-10, 64 u N / min_gap),
 *                  u = 2^-53, at most 1e-6), P S P is squared again until some of
 *                  them decay, and those move to the complement (at most three
 *                  rounds).  Squarings stop at 2^m with m <= log2(0.02 / (u sqrt N))
 *                  (40 to 44 for N = 16384 .. 64), where FP64 drift of an exact -1
 *                  eigenvalue would become visible.  The call refuses
 *                  (FGFRFT_ERR_AMBIGUOUS_SPECTRUM) a spectrum it cannot certify: an
 *                  eigenvalue left in the complement closer than 1e-6 to -1
 *                  (min_gap below), or a counted set that cannot be separated
 *                  within the squaring limit (|lambda + 1| between about 1e-10 and
 *                  2e-6).
 *               in [1e-5, 0.5]: fixed threshold.  S is squared exactly
 *                  ceil(log2(4 ln 2 / neg1_tol^2)) times, which takes an eigenvalue
 *                  with |lambda + 1| = neg1_tol to at most 1/2; eigenvalues below
 *                  about 0.28 x that boundary count as -1, those above about 2.06 x
 *                  it do not (the boundary lies in (neg1_tol / sqrt 2, neg1_tol]),
 *                  and one in between returns FGFRFT_ERR_AMBIGUOUS_SPECTRUM.
 *               Any other value: FGFRFT_ERR_INVALID_ARG.  Ignored with W_dev.
 *   P_dev       optional N x N complex128 device output: the FP64 projector P
 *               before it is rounded into storage (16-byte aligned; NULL: not
 *               written).
 *   plan_mem    device buffer of at least fgfrft_plan_bytes(N, L_max, storage)
 *               bytes, 256-byte aligned; it holds the plan for its lifetime.
 *   work        device scratch of fgfrft_precompute_work_bytes(N) bytes,
 *               256-byte aligned; free again when the call returns.
 *   out         receives the plan handle (a small host record; release it
 *               with fgfrft_plan_destroy).
 * Checks ||F^H F - I||_F / sqrt(N) <= 1e-8 (FGFRFT_ERR_NOT_UNITARY).  A real F
 * (every imaginary part exactly 0, no W) is processed with real FP64 products.
 * Synchronises the stream (it reads traces back to the host).
 */
int fgfrft_precompute(const double* F_dev, int64_t N, int L_max, int storage,
                      const double* W_dev, int64_t r_W, double neg1_tol, double* P_dev,
                      void* plan_mem, size_t plan_bytes,
                      void* work, size_t work_bytes,
                      void* stream, fgfrft_plan* out);

/* Plan metadata; any output pointer may be NULL.
 *   r_neg1         rank of P (the multiplicity of lambda = -1).
 *   proj_residual  ||F P + P||_F after precompute (0 when r_neg1 = 0); for the
 *                  exact projector it is sqrt(sum over the counted eigenvalues of
 *                  |lambda_k + 1|^2).
 *   squarings      squaring steps the projector needed (0 when W was given).
 *   min_gap        two doubles: a lower and an upper bound of
 *                  min_{k not in I_-1} |lambda_k + 1| = 2 cos_{c,min} (the distance
 *                  of the nearest complementary eigenvalue from -1, Thm. 2), from
 *                  the traces of repeated squares of the complement part of S;
 *                  upper / lower <= 1.01 unless the 2^52-th power was reached
 *                  first; both +inf when every eigenvalue is -1. */
int fgfrft_plan_info(fgfrft_plan p, int64_t* N, int* L_max, int* storage, int* r_neg1,
                     double* proj_residual, int* squarings, size_t* plan_bytes, double* min_gap);

/* Device pointer to stored block l (-L_max <= l <= L_max, or l = L_max + 1 for
 * P) in the given storage (one bit), and the element stride between blocks.
 * For FGFRFT_STORE_C64 the block is N x N c64; for FGFRFT_STORE_SPLIT_F16 it is
 * four consecutive fp16 planes of N rows of pitch round_up(N, 8); for
 * FGFRFT_STORE_HALF the two tiled FP32 planes described there.  NULL if absent
 * (a negative l in FGFRFT_STORE_HALF). */
const void* fgfrft_plan_block(fgfrft_plan p, int storage, int l, int64_t* block_stride_elems);

/* Synchronise the stream, read the plan's device status word and clear it:
 * FGFRFT_OK, or FGFRFT_ERR_TIMEOUT when a kernel's bounded wait ran out. */
int fgfrft_plan_status(fgfrft_plan p, void* stream);

/* 1 if F was real (all imaginary parts exactly 0) and no W was supplied: every stored
 * block is then real and the tensor-core paths skip the imaginary planes (6 instead of
 * 12 MMAs per k16 step; the skipped products are exact zeros).  0 otherwise;
 * -FGFRFT_ERR_INVALID_ARG for a NULL plan. */
int fgfrft_plan_real(fgfrft_plan p);

/* 1 if the plan holds the pair stack: F real with no eigenvalue -1 (r_-1 = 0),
 * FGFRFT_STORE_ENTRY_F16, N a multiple of 128, L_max a multiple of 16 and the pair launch
 * fits in the device's shared memory (L_max <= 64 on GB300).
 * Then M_{-l} = M_l^T (F^{-1} = F^T; Prop. 2) and M_0 = P_c = I, so the fused multi-order
 * assembly of split operators (the assembled path of fgfrft_apply) reads one row of the
 * 2 L_max powers l != 0 per entry pair {(i, k), (k, i)} (i/128 <= k/128), about half the
 * bytes of the full entry-major copy, and forms Q[i][k] and Q[k][i] from it (Def. 1 with
 * c_{-l} for the mirror).  The pair stack occupies the entry-major storage's imaginary
 * planes, which a real F leaves unused, so the plan size does not change.  0 otherwise;
 * -FGFRFT_ERR_INVALID_ARG for a NULL plan. */
int fgfrft_plan_pair(fgfrft_plan p);

/* Release the host record of a plan.  Frees nothing caller-owned. */
int fgfrft_plan_destroy(fgfrft_plan p);

/* Bytes of scratch an online call needs (op = enum fgfrft_op).  count is A
 * for FGFRFT_OP_ASSEMBLE and B otherwise; alpha_host is needed because the
 * assembled path sizes its scratch by the number of distinct orders. */
size_t fgfrft_work_bytes(fgfrft_plan p, int op, const double* alpha_host, int64_t count,
                         int L, int flags);

/*
 * Online part of Algorithm 1 (Def. 1), A orders in one pass over the stack.
 *   alpha_host  A orders.
 *   Q_dev       A x N x N c64 output, Q_dev[a][i][k] = (Q_L^{alpha_a})_{ik}.
 * A = 1 streams the stored blocks once: the L + 2 half-stack blocks as pairs
 * of transposed tiles with FGFRFT_STORE_HALF, else the 2L + 2 c64 blocks
 * (the two real split planes for a real F) with bulk-copy staging.  A > 1
 * without an entry-major copy repeats that per order.  A > 1 reads each stored entry once for all A
 * outputs: as one tensor-core GEMM over the entry-major split stack when the plan
 * has FGFRFT_STORE_ENTRY_F16 (split-fp16 products, FP32 accumulation), else on
 * FP32 CUDA cores from the c64 stack.
 */
int fgfrft_assemble(fgfrft_plan p, const double* alpha_host, int64_t A, int L,
                    void* Q_dev, void* work, size_t work_bytes, void* stream);

/*
 * Y[:, j] = Q_L^{alpha_j} X[:, j] for j = 0..B-1 (Def. 2), or (Q_L^{alpha_j})^H X[:, j]
 * with FGFRFT_ADJOINT.
 *   alpha_host  B orders, or 1 with FGFRFT_SHARED_ALPHA.
 *   X_dev, Y_dev  B x N c64 (signal j at offset j * N).
 * Path: the FGFRFT_PATH_* bit in flags, else chosen by the library: columns
 * are grouped into runs of equal order; runs of at least 64 columns use
 * FGFRFT_PATH_ASSEMBLED, otherwise FGFRFT_PATH_STACKED (tensor paths need
 * FGFRFT_STORE_SPLIT_F16, else the FP32 paths are used).
 * FGFRFT_REAL_SIGNALS / FGFRFT_REAL_OUTPUT take real float32 signals / outputs
 * (half the bytes; FGFRFT_ERR_UNSUPPORTED where their conditions do not hold).
 */
int fgfrft_apply(fgfrft_plan p, const double* alpha_host, int64_t B, int L,
                 const void* X_dev, void* Y_dev, int flags,
                 void* work, size_t work_bytes, void* stream);

/*
 * Forward with dual accumulators and the backward of Y = Q_L^{alpha_j} X[:, j].
 * Forward (X_dev != NULL): Y (if Y_dev) and D = dY/dalpha (if dY_dev, Prop. 3)
 *   from the same pass over the stored powers.
 * Backward (G_dev != NULL), G = dloss/dRe(Y) + j dloss/dIm(Y):
 *   gradX = (Q_L^{alpha_j})^H G[:, j] (if gradX_dev; Prop. 2), and
 *   gradalpha[j] = Re sum_i conj(G_ij) D_ij (if gradalpha_dev), with D read
 *   from dY_dev (computed in this call or an earlier one).  With
 *   FGFRFT_SHARED_ALPHA (alpha_host holds one order for every column) the
 *   gradient of that one order is written: gradalpha[0] = sum_j of the above
 *   (FP64 partial sums added in a fixed order, one float written).
 * Paths: FGFRFT_PATH_STACKED (default with FGFRFT_STORE_SPLIT_F16) or
 * FGFRFT_PATH_STACKED_FP32.
 */
int fgfrft_grad(fgfrft_plan p, const double* alpha_host, int64_t B, int L,
                const void* X_dev, void* Y_dev, void* dY_dev,
                const void* G_dev, void* gradX_dev, float* gradalpha_dev,
                int flags, void* work, size_t work_bytes, void* stream);

/* Kernel classes for launch counting and timing. */
enum fgfrft_kernel_class {
  FGFRFT_KC_COEFFS = 0,          /* per-column coefficients (FP64 on the device) */
  FGFRFT_KC_ASSEMBLE_SINGLE = 1, /* one-order assembly, bulk-copy streaming */
  FGFRFT_KC_ASSEMBLE_MULTI = 2,  /* fused multi-order assembly (CUDA-core or tensor-core kernel) */
  FGFRFT_KC_SPLIT_SIGNALS = 3,   /* fp16 hi/lo split of signal columns */
  FGFRFT_KC_TC_GEMM = 4,         /* tcgen05 stacked / grouped GEMM */
  FGFRFT_KC_SIMT_GEMM = 5,       /* FP32 CUDA-core GEMM */
  FGFRFT_KC_GRAD_REDUCE = 6,     /* alpha-gradient reduction */
  FGFRFT_KC_OFFLINE = 7,         /* FP64 offline kernels */
  FGFRFT_KC_COUNT = 8
};

/* Process-wide instrumentation.  Launch counts are always kept.  While timing is
 * enabled, every call that launches kernels of a class records a CUDA event pair
 * around those launches on the call's stream (at most 65536 pairs per class
 * between resets).  Enabling creates a pool of 512 event pairs per class, so that timed
 * calls only record events.  fgfrft_timing_read synchronises on the recorded events and
 * returns the launches, the timed calls and the summed device time in ms. */
int fgfrft_timing_enable(int on);
int fgfrft_timing_reset(void);
int fgfrft_timing_read(int kernel_class, int64_t* launches, int64_t* timed_calls, double* total_ms);

/* Failure-path check: launches one CTA whose bounded device wait (the helper every
 * kernel uses, limit 2 s) waits on an mbarrier that nothing completes.  The wait runs
 * out, FGFRFT_ERR_TIMEOUT is recorded in the plan's status word exactly as for a stalled
 * kernel (read and cleared by fgfrft_plan_status), and the kernel returns; nothing faults
 * and the context stays usable.  For tests of the error path.  No counterpart in the
 * paper. */
int fgfrft_check_wait_timeout(fgfrft_plan p, void* stream);

/*
 * Zero-allocation alpha-gradient: gradalpha[j] = Re sum_i conj(G_ij) D_ij for
 * j < B, the same quantity fgfrft_grad returns in gradalpha_dev, for callers that
 * cannot allocate device memory when they need it (code inside an allocator or
 * a real-time section where cudaMalloc and cudaFree, which synchronise the
 * device, are not allowed, or a host that only passes its input
 * and output buffers).  The paper has no counterpart: this is an interface
 * choice of the library.
 *   G_dev, D_dev    B x N c64 (signal j at offset j * N): the output gradient
 *                   and dY/dalpha from fgfrft_grad's forward.
 *   gradalpha_dev   B floats, written.
 * The FP64 partial sums (one per signal and 1024-entry chunk) live in a fixed
 * array of FGFRFT_NOALLOC_MAX_PARTIALS doubles (512 KiB) in the library's device
 * memory, which every GPU that loads the library holds until the process exits.
 * Requests with B * ceil(N / 1024) > FGFRFT_NOALLOC_MAX_PARTIALS return
 * FGFRFT_ERR_UNSUPPORTED before anything is enqueued.  The call allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine.  Its first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and keeps it for the life of the process.  A cudaDeviceReset (or any other teardown of the
 * device's primary context) invalidates the kept address: do not call this entry
 * point on a device after resetting it in the same process.  All calls
 * share the one array and every call overwrites the part it uses, so calls that
 * overlap on the GPU (different streams without ordering) race.
 */
#define FGFRFT_NOALLOC_MAX_PARTIALS 65536
int fgfrft_grad_alpha_noalloc(const void* G_dev, const void* D_dev, int64_t B, int64_t N,
                              float* gradalpha_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FGFRFT_H */
