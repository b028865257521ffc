/*
 * ptdr.h -- C ABI of libptdr, a GB300 (sm_103a) library for the Pauli
 * decomposition of Koska, Baboulin and Gazda, "A tree-approach Pauli
 * decomposition algorithm with application to quantum computing"
 * (arXiv 2403.11644, "PTDR").
 *
 * What is computed (Sec. II.A, "Decomposition in the Pauli operator basis"
 * and "Straightforward decomposition method"): for a complex 2^n x 2^n
 * matrix A, all 4^n coefficients
 *
 *     c_P = 2^-n tr(P A),   P = sigma_{n-1} (x) ... (x) sigma_0,
 *
 * so that A = sum_P c_P P.  Operators are labelled with the paper's
 * PauliComposer notation (Sec. II.B): qubit l <-> bit l of a row/column
 * index, and P <-> two n-bit masks (x, z) with x_l = d(sigma_l) (1 for X and
 * Y, the diagonality function) and z_l = 1 for Y and Z.  P_{x,z} has one
 * nonzero per row j, at column j XOR x (Sec. II.A, "First optimization of
 * the trace computation").
 *
 * Layouts (all row-major, complex numbers interleaved re, im):
 *   A  : A[r * 2^n + c]                                     (2^n x 2^n)
 *   C  : C[x * 2^n + z] = c_{P(x,z)}                        (4^n values)
 *   band storage (Sec. IV.A, diagonal/tridiagonal/band-diagonal matrices):
 *        bands[(d + s) * 2^n + c] = A[c + d][c],  d in [-s, s];
 *        slots whose row c + d falls outside the matrix are ignored.
 *
 * Conventions shared by every entry point:
 *   - All data pointers are DEVICE pointers owned by the caller, except the
 *     arguments explicitly named h_* (host).  The library never allocates
 *     device memory on these paths; scratch space is the caller-provided
 *     workspace, whose size is queried first.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  Argument errors are returned synchronously before
 *     anything is enqueued.  Errors detected on the device (a bounded wait
 *     that ran out, an index check in a checked build) are recorded in a
 *     device status word read by ptdr_last_device_status().
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     call returns PTDR_ERR_NO_DEVICE.
 *   - Inputs and outputs must not overlap.  Pointers must be aligned to
 *     their element size (16 bytes for complex types is recommended; the
 *     vectorised paths need it and fall back to narrower loads otherwise).
 */
#ifndef PTDR_H
#define PTDR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PTDR_OK = 0,
    PTDR_ERR_INVALID_ARG = 1, /* null pointer, bad n/s/count, bad enum value, overlap */
    PTDR_ERR_UNSUPPORTED = 2, /* valid but unsupported dtype/precision combination */
    PTDR_ERR_NO_DEVICE = 3,   /* no CUDA device or driver; nothing was run */
    PTDR_ERR_CUDA = 4,        /* a CUDA runtime call failed (launch, copy, attribute) */
    PTDR_ERR_WORKSPACE = 5,   /* workspace null or smaller than the queried size */
    PTDR_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    PTDR_ERR_INTERNAL = 7     /* device-side consistency check failed */
} ptdr_status;

typedef enum {
    PTDR_C64 = 0,  /* complex float  (re, im float32) */
    PTDR_C128 = 1, /* complex double (re, im float64) */
    PTDR_F32 = 2,  /* real float32 */
    PTDR_F64 = 3   /* real float64 */
} ptdr_dtype;

typedef enum {
    /* float64 arithmetic on the FP64 pipe (full-accuracy mode) */
    PTDR_PREC_FP64 = 0,
    /* float32 arithmetic on the CUDA cores */
    PTDR_PREC_FP32 = 1,
    /* Hadamard stages as dense +-1 tensor-core tiles on bf16 hi/mid/lo splits
       of float32 data, accumulated in float32 (the +-1 matrix is exact in bf16) */
    PTDR_PREC_SPLIT_BF16_TC = 2,
    /* exact transform in 128-bit two's-complement fixed point on the integer
       pipe: the input is rounded once to 2^-(124-n) of its largest magnitude
       (one shared exponent from a pre-pass), every butterfly is an exact
       integer add, and each result is rounded once to the output type, so the
       result has FP64 accuracy without the FP64 pipe (dense decompose and
       compose; inputs must be finite) */
    PTDR_PREC_FIXED_I128 = 3
} ptdr_precision;

typedef enum {
    PTDR_OP_DECOMPOSE = 0,
    PTDR_OP_COMPOSE = 1
} ptdr_op;

/*
 * ptdr_decompose -- all 4^n coefficients of a dense matrix.
 * Defines: c_P = 2^-n tr(P A) for every P in P_n (Sec. II.A; the paper's
 * Algorithm 1 computes the same set by walking the Pauli tree, Sec. III.A).
 *
 *   A, a_type   device, 4^n elements of a_type, row-major: C64, C128, or a
 *               real matrix (F32, F64).
 *   C, c_type   device, 4^n elements of c_type; C[x*2^n + z].  C64 / C128
 *               store c_P; a real type (F32 / F64) stores Re c_P only, which
 *               for a Hermitian A is all of c_P (Thm 2: Hermitian matrices
 *               have real coefficients) -- the Hermitian real-output mode,
 *               half the write bytes of a complex output.
 *   n           1 <= n <= 15.
 *   prec        FP64: any a_type/c_type.  FP32: any a_type/c_type (C128 input
 *               is rounded to float32 on load).  SPLIT_BF16_TC: n = 14,
 *               a_type = C64, c_type = C64 or F32, with A, C and the workspace 32-byte
 *               aligned (PTDR_ERR_INVALID_ARG otherwise); other n or types
 *               return PTDR_ERR_UNSUPPORTED.  FIXED_I128: any a_type/c_type
 *               (a non-finite input entry is recorded as PTDR_ERR_INVALID_ARG
 *               in the device status word and the output is then undefined).
 *   workspace   device scratch of at least ptdr_workspace_size() bytes (may
 *               be NULL when that size is 0).
 * Returns PTDR_OK once the work is enqueued on `stream`.
 */
ptdr_status ptdr_decompose(const void* A, ptdr_dtype a_type, void* C, ptdr_dtype c_type, int n,
                           ptdr_precision prec, void* workspace, size_t workspace_bytes,
                           void* stream);

/*
 * ptdr_compose -- the inverse map: A = scale * sum_P c_P P.
 * Defines: the expansion A = sum_P alpha_P P of Sec. II.A.  With scale = 1 it
 * rebuilds A from ptdr_decompose's output; with scale = 2^-n it is the
 * adjoint of ptdr_decompose (D(A)_P = 2^-n <P, A>), which is the backward
 * pass of the decomposition for automatic differentiation.
 *
 *   C, c_type   device, 4^n coefficients: C64, C128, or real coefficients
 *               (F32, F64), which describe a Hermitian A (Thm 2).
 *   A, a_type   device output, 4^n elements, a_type in {C64, C128}.
 *   n, prec, workspace, stream as for ptdr_decompose (SPLIT_BF16_TC unsupported;
 *               FIXED_I128 applies a power-of-two scale exactly and any
 *               other scale with one final FP64 multiply).
 */
ptdr_status ptdr_compose(const void* C, ptdr_dtype c_type, void* A, ptdr_dtype a_type, int n,
                         double scale, ptdr_precision prec, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * ptdr_workspace_size -- device scratch bytes needed by ptdr_decompose or
 * ptdr_compose for (n, a_type, c_type, prec).  Host only; no CUDA call.
 */
ptdr_status ptdr_workspace_size(ptdr_op op, int n, ptdr_dtype a_type, ptdr_dtype c_type,
                                ptdr_precision prec, size_t* bytes);

/*
 * ptdr_structured_masks -- the X/Z-flip masks x that a band-diagonal matrix
 * of half-width s can populate (s = 0: diagonal, s = 1: tridiagonal).
 * Defines: Sec. IV.A.1 (diagonal: only I/Z terms, i.e. x = 0), Thm 3
 * (tridiagonal: at most (n+1) 2^n terms) and Thm 4 (band-diagonal: at most
 * (s n - c(s)) 2^n terms).  A mask x != 0 with highest set bit h is reachable
 * iff 2^h - (x mod 2^h) <= s (the smallest |row - column| over the entries of
 * the XOR-diagonal x).  Host only; no CUDA call.
 *
 *   n          1 <= n <= 40.   s >= 0.
 *   h_masks    host output, ascending; may be NULL to query the count.
 *   count      in: capacity of h_masks (ignored when h_masks is NULL);
 *              out: number of masks.  Returns PTDR_ERR_INVALID_ARG if the
 *              capacity is too small (count then holds the number needed).
 */
ptdr_status ptdr_structured_masks(int n, int s, uint64_t* h_masks, size_t* count);

/*
 * ptdr_decompose_structured -- the coefficients of a band-diagonal matrix on
 * the given masks only (the paper prunes the X/Y subtrees, Sec. IV.A; here
 * only the listed XOR-diagonals are gathered and transformed).
 *
 *   bands, b_type  device band storage (see layout above), (2s+1) * 2^n
 *                  elements of b_type in {F32, F64, C64, C128}.
 *   n, s           1 <= n <= 30, 0 <= s < 2^n.
 *   h_masks        HOST array of n_masks masks (each < 2^n), e.g. from
 *                  ptdr_structured_masks(); the launches are planned from it,
 *                  so a mask list costs no device-side table.
 *   C, c_type      device output, n_masks * 2^n elements; row i holds mask
 *                  h_masks[i]: C[i * 2^n + z].  c_type complex, or real
 *                  (F32/F64) for a real symmetric band input, whose
 *                  coefficients are real (Thm 2): the real part is stored.
 *   prec           FP64 or FP32.
 *   workspace      at least ptdr_structured_workspace_size() bytes.
 */
ptdr_status ptdr_decompose_structured(const void* bands, ptdr_dtype b_type, int n, int s,
                                      const uint64_t* h_masks, size_t n_masks, void* C,
                                      ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                      size_t workspace_bytes, void* stream);

/* Workspace bytes for ptdr_decompose_structured.  Host only. */
ptdr_status ptdr_structured_workspace_size(int n, int s, const uint64_t* h_masks, size_t n_masks,
                                           ptdr_dtype b_type, ptdr_dtype c_type,
                                           ptdr_precision prec, size_t* bytes);

/*
 * Anti-band matrices (Remark 1 of Sec. IV.A: for anti-diagonal matrices the
 * roles of I, Z and of X, Y swap).  A is anti-band of half-width s when
 * A[r][c] = 0 unless |r + c - (2^n - 1)| <= s (s = 0: anti-diagonal).  Then
 * B = A J, J = X (x) ... (x) X the exchange matrix, is band-diagonal, and the
 * anti-band storage is B's band storage:
 *        antibands[(d + s) * 2^n + c] = A[c + d][2^n - 1 - c],  d in [-s, s].
 * The reachable masks are the band's masks XOR (2^n - 1) (anti-diagonal: the
 * single mask x = 2^n - 1, only X and Y on every qubit), and the coefficient
 * of mask x_A is (-1)^{|z|} (-i)^{|x_A & z|} 2^-n WHT(d_{x_A ^ (2^n - 1)})[z]
 * over B's gathered diagonal.
 *
 * ptdr_antistructured_masks -- as ptdr_structured_masks, for anti-band masks
 *   (ascending).  Host only.
 * ptdr_decompose_antistructured -- as ptdr_decompose_structured, with the
 *   anti-band storage above and anti-band masks in h_masks; row i of C holds
 *   mask h_masks[i].  A real output type stores the real part (all of c when
 *   A is Hermitian, Thm 2).
 * ptdr_antistructured_workspace_size -- its workspace bytes.  Host only.
 */
ptdr_status ptdr_antistructured_masks(int n, int s, uint64_t* h_masks, size_t* count);
ptdr_status ptdr_decompose_antistructured(const void* antibands, ptdr_dtype b_type, int n, int s,
                                          const uint64_t* h_masks, size_t n_masks, void* C,
                                          ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                          size_t workspace_bytes, void* stream);
ptdr_status ptdr_antistructured_workspace_size(int n, int s, const uint64_t* h_masks, size_t n_masks,
                                               ptdr_dtype b_type, ptdr_dtype c_type,
                                               ptdr_precision prec, size_t* bytes);

/*
 * Matrix-free input (Sec. V.B: the decomposition does not need the input
 * stored when its entries can be computed, e.g. from a function).
 *
 * The masks are processed in x-blocks of 2^a, a = min(7, n).  Block xt
 * (masks xt 2^a .. xt 2^a + 2^a - 1) reads exactly the sheared tile set
 *     S[i * 2^n + k] = A[(((k >> a) ^ xt) << a) + i][k],   i < 2^a, k < 2^n,
 * (the 2^a x 2^a tiles (cb ^ xt, cb) of A, one per column block cb), and every
 * tile of A belongs to exactly one block.  Before each block the library calls
 * fill(user, n, xt, a, d_S, stream), which must enqueue on `stream` (or
 * finish before returning) the writes of S into the device buffer d_S
 * (2^a x 2^n elements of a_type, row-major) and return 0; a nonzero return
 * stops the call with PTDR_ERR_INTERNAL.  The device then holds 2^a rows of A
 * at a time instead of 2^n, and each entry is produced once.  fill runs on the
 * calling thread, blocks in ascending xt.
 */
typedef int (*ptdr_tile_fn)(void* user, int n, uint64_t x_tile, int a, void* d_S, void* stream);

/*
 * ptdr_decompose_matrix_free -- ptdr_decompose with A produced block by block
 * by `fill` (above).  n, a_type, C, c_type as for ptdr_decompose; prec FP64 or
 * FP32 (generic tile kernels); workspace (256-byte aligned) of at least
 * ptdr_matrix_free_workspace_size() bytes holds S and, for rows longer than
 * one tile, the block's intermediate rows.
 */
ptdr_status ptdr_decompose_matrix_free(int n, ptdr_dtype a_type, ptdr_tile_fn fill, void* user, void* C,
                                       ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                       size_t workspace_bytes, void* stream);

/* Workspace bytes for ptdr_decompose_matrix_free.  Host only. */
ptdr_status ptdr_matrix_free_workspace_size(int n, ptdr_dtype a_type, ptdr_dtype c_type,
                                            ptdr_precision prec, size_t* bytes);

/*
 * ptdr_decompose_batched -- decomposes `count` independent matrices of
 * possibly different sizes in one persistent launch (the paper's forest of
 * independent subtrees, Sec. V.B, taken across matrices).
 *
 *   d_A      device array of `count` device pointers to the inputs.
 *   d_C      device array of `count` device pointers to the outputs.
 *   d_n      device array of `count` sizes n_i.
 *   h_n      the same sizes on the host (sizes the grid and workspace).
 *   count    >= 1.  1 <= n_i <= 13.
 *   a_type, c_type, prec as for ptdr_decompose (FP32 or FP64).
 *   workspace at least ptdr_batched_workspace_size() bytes.
 * The launch sequence is fixed for a given h_n, so it can be captured in a
 * CUDA graph and replayed with new data behind the same pointers.
 */
ptdr_status ptdr_decompose_batched(const void* const* d_A, void* const* d_C, const int* d_n,
                                   const int* h_n, int count, ptdr_dtype a_type,
                                   ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                   size_t workspace_bytes, void* stream);

/* Workspace bytes for ptdr_decompose_batched.  Host only. */
ptdr_status ptdr_batched_workspace_size(const int* h_n, int count, ptdr_dtype a_type,
                                        ptdr_dtype c_type, ptdr_precision prec, size_t* bytes);

/*
 * ptdr_decompose_batched_static -- ptdr_decompose_batched for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is a
 * library convenience, not part of the method.
 *
 * Who needs it: an application that embeds this library but owns all device
 * memory through its own pool, code on a latency-critical stream where an
 * allocation would synchronise the device, or a runtime that forbids
 * allocations after start-up.  Such a caller
 * cannot provide the workspace ptdr_decompose_batched asks for.  This variant
 * allocates nothing: its scratch is a fixed 32,784-byte array in the library's
 * device image (every GPU that loads the library holds it until exit).
 *
 *   Arguments as for ptdr_decompose_batched, without the workspace.
 *   count      at most 4096 matrices; larger batches return
 *              PTDR_ERR_WORKSPACE (use ptdr_decompose_batched instead).
 *   The first call on each device looks up the array's device address (with
 *   that device current) and caches it for the life of the process; do not use
 *   the library across a cudaDeviceReset (which reloads the array at a new
 *   address).  Every call shares the one array, which keeps the last
 *   call's tables; each call rewrites all of it (including the work-queue
 *   counter) before use, so results never depend on an earlier call, but two
 *   calls whose work overlaps on the GPU (different streams, or different
 *   host threads without ordering) race on it and must not be issued.
 */
ptdr_status ptdr_decompose_batched_static(const void* const* d_A, void* const* d_C,
                                          const int* d_n, const int* h_n, int count,
                                          ptdr_dtype a_type, ptdr_dtype c_type,
                                          ptdr_precision prec, void* stream);

/*
 * ptdr_decompose_host -- ptdr_decompose for matrices held in HOST memory.
 * Defines: the same coefficients as ptdr_decompose (Sec. II.A), for `count`
 * independent matrices; the host buffers are copied in and out by the call.
 *
 *   h_A       host array of `count` host pointers to the inputs (4^n elements
 *             of a_type each, row-major); page-locked memory (cudaHostAlloc /
 *             cudaHostRegister) lets the copies overlap, pageable memory is
 *             accepted but its copies do not overlap.
 *   h_C       host array of `count` host pointers to the outputs (4^n
 *             elements of c_type each).
 *   count     >= 1.
 *   a_type, c_type, n, prec as for ptdr_decompose.
 *   d_scratch device memory of at least ptdr_decompose_host_scratch_size()
 *             bytes, 256-byte aligned: two input buffers, two output buffers
 *             and the decomposition workspace (the library allocates nothing).
 * The upload of matrix i + 1, the decomposition of matrix i and the download
 * of matrix i - 1 run concurrently (two library-owned streams per device,
 * ordered by events).  All work follows what was enqueued on `stream` before
 * the call, and `stream` completes after the last download: synchronise it
 * before reading h_C.  Calls from several host threads are enqueued one at a
 * time.  Argument errors are returned before anything is enqueued.
 */
ptdr_status ptdr_decompose_host(const void* const* h_A, void* const* h_C, int count, ptdr_dtype a_type,
                                ptdr_dtype c_type, int n, ptdr_precision prec, void* d_scratch,
                                size_t d_scratch_bytes, void* stream);

/* Device scratch bytes for ptdr_decompose_host.  Host only. */
ptdr_status ptdr_decompose_host_scratch_size(int n, ptdr_dtype a_type, ptdr_dtype c_type,
                                             ptdr_precision prec, size_t* bytes);

/*
 * Autotuner of the strided HBM passes.  Rows too long for one on-chip tile
 * (FP64 n >= 14, complex128 input at n = 15, compose n = 15, ...) run as a
 * first pass over row segments and strided passes over the high bits of the
 * transform through an intermediate in HBM -- the GPU form of the forest cut
 * at a level of Sec. V.B.  Their schedule is a tuning choice.
 */
typedef struct {
    int tile_log2;      /* first-pass tile, log2 of its bytes (15..17) */
    int masks_log2;     /* masks per first-pass tile, log2 (0..3; 0 for compose) */
    int pass_tile_log2; /* strided-pass tile, log2 bytes: sets the bits per pass */
    int threads;        /* threads per CTA (256 or 512) */
    double ms;          /* the measured time of one call with this schedule */
} ptdr_tune_params;

/*
 * ptdr_autotune -- times every candidate schedule of the multi-pass plan of
 * ptdr_decompose (op = PTDR_OP_DECOMPOSE) or ptdr_compose (PTDR_OP_COMPOSE)
 * for (n, in_type, out_type, prec) with CUDA events on `stream`, on the
 * caller's buffers (in is read, out and the workspace are overwritten), and
 * keeps the fastest for this GPU: in memory, and in the JSON file that the
 * environment variable PTDR_TUNE_CACHE names, if any.  Synchronous (it waits
 * for its timings).  Later calls of ptdr_decompose / ptdr_compose with the
 * same GPU, op, n, types and precision run the stored schedule.  Returns
 * PTDR_ERR_UNSUPPORTED when the plan has no strided passes (rows fit on chip,
 * or a dedicated kernel runs them); arguments as for ptdr_decompose.
 */
ptdr_status ptdr_autotune(ptdr_op op, int n, ptdr_dtype in_type, ptdr_dtype out_type,
                          ptdr_precision prec, const void* in, void* out, void* workspace,
                          size_t workspace_bytes, void* stream, ptdr_tune_params* best);

/*
 * ptdr_tune_lookup / ptdr_tune_store -- host-only access to the tuning cache
 * (loaded lazily from PTDR_TUNE_CACHE).  The key is the GPU name as
 * cudaGetDeviceProperties reports it, the op, n, the two types and the
 * precision.  Lookup returns PTDR_ERR_UNSUPPORTED when the key has no entry;
 * store replaces the entry and rewrites the file (PTDR_ERR_INVALID_ARG if it
 * cannot be written).
 */
ptdr_status ptdr_tune_lookup(const char* gpu_name, ptdr_op op, int n, ptdr_dtype in_type,
                             ptdr_dtype out_type, ptdr_precision prec, ptdr_tune_params* out);
ptdr_status ptdr_tune_store(const char* gpu_name, ptdr_op op, int n, ptdr_dtype in_type,
                            ptdr_dtype out_type, ptdr_precision prec, const ptdr_tune_params* params);

/*
 * ptdr_last_device_status -- synchronises `stream`, returns the status word
 * the kernels wrote since the previous call (PTDR_OK if none) and clears it.
 */
ptdr_status ptdr_last_device_status(void* stream);

/*
 * Decomposition algebra (Sec. IV.B, "Combinations of matrices"): the
 * decomposition of a matrix built from others, computed from their
 * coefficient arrays (layout C[x*2^n + z]) without decomposing it again.
 * Device pointers; asynchronous on `stream`; the library allocates nothing.
 */

/*
 * ptdr_coeff_lincomb -- linear combination (Sec. IV.B.3): the coefficients of
 * mu A + B are mu alpha_j + beta_j.  C_out = mu * CA + CB elementwise.
 *   n          1 <= n <= 15 (4^n coefficients per array).
 *   mu_re, mu_im  the complex factor mu (real arrays need mu_im = 0:
 *              PTDR_ERR_UNSUPPORTED otherwise).
 *   CA, CB     device inputs of c_type; CB may be NULL (C_out = mu CA).
 *   C_out      device output of c_type; may be CB itself (in place), must not
 *              otherwise overlap an input.
 *   c_type     C64, C128 (computed in float32 / float64), F32, F64.
 */
ptdr_status ptdr_coeff_lincomb(int n, double mu_re, double mu_im, const void* CA, const void* CB,
                               void* C_out, ptdr_dtype c_type, void* stream);

/*
 * ptdr_coeff_block_diag -- direct sum and block-diagonal matrices (Sec.
 * IV.B.1-2).  The block-diagonal matrix diag(A_0, ..., A_{2^m - 1}) of 2^m
 * blocks of n qubits is sum_i |i><i| (x) A_i, and |i><i| =
 * 2^-m sum_t (-1)^{|t & i|} Z^t on the top m qubits, so its n + m qubit
 * coefficients are
 *     C_out[x][z + 2^n t] = 2^-m sum_i (-1)^{|t & i|} C_i[x][z]   (x < 2^n),
 * and 0 for every mask x >= 2^n (no X or Y on a top qubit).  m = 1 is the
 * direct sum A (+) B = I (x) (A + B)/2 + Z (x) (A - B)/2; larger block
 * counts follow by applying it to groups (the paper's recursive pairing).
 *   n, m       n >= 1, 1 <= m <= 4, n + m <= 15.
 *   h_blocks   HOST array of 2^m device pointers: block i's coefficients (4^n
 *              of c_type), block i sits at rows/columns [i 2^n, (i+1) 2^n).
 *   C_out      device output, 4^(n+m) coefficients of c_type, 16-byte aligned,
 *              not overlapping a block.
 */
ptdr_status ptdr_coeff_block_diag(int n, int m, const void* const* h_blocks, void* C_out,
                                  ptdr_dtype c_type, void* stream);

/*
 * ptdr_coeff_hermitian_augment -- Hermitian matrix augmentation (Sec.
 * IV.B.5): [[0, A^H], [A, 0]] = X (x) sum Re(alpha_j) P_j + Y (x) sum
 * Im(alpha_j) P_j, so on n + 1 qubits
 *     C_out[x + 2^n][z] = Re CA[x][z],   C_out[x + 2^n][z + 2^n] = Im CA[x][z],
 * and every other coefficient is 0.  All are real (the augmented matrix is
 * Hermitian, Thm 2); at most twice as many nonzero terms as A has.
 *   CA, a_type      device, 4^n coefficients (C64, C128; F32/F64 = real).
 *   C_out, out_type device, 4^(n+1) coefficients, 16-byte aligned: real
 *                   (F32, F64) or complex (C64, C128, zero imaginary parts).
 *   n               1 <= n <= 14.
 */
ptdr_status ptdr_coeff_hermitian_augment(int n, const void* CA, ptdr_dtype a_type, void* C_out,
                                         ptdr_dtype out_type, void* stream);

/*
 * ptdr_coeff_select -- the sparse form of a decomposition that a block-encoding
 * by a linear combination of unitaries needs (Sec. VI, "Block-encoding using
 * Pauli decomposition"): the kept terms P_i, their coefficients alpha_i and
 * the normaliser sum_i |alpha_i| of the ancilla state
 * sum_i sqrt(|alpha_i|) |i> / sqrt(sum_i |alpha_i|).
 * Keeps every coefficient with |c_P| > threshold; with k > 0, only the k
 * largest of those (ties in magnitude go to the lower index x*2^n + z).
 * Magnitudes are compared in float32 for complex64/float32 arrays and as
 * |c|^2 in float64 for complex128 (so complex128 values below about 1e-154
 * count as zero); float64 arrays compare |v|.
 *   n            1 <= n <= 15; C holds 4^n coefficients of c_type (any type).
 *   threshold    finite, >= 0 (0 keeps every nonzero coefficient).
 *   k            0 = no count limit.
 *   d_idx, d_val device outputs, capacity `cap` each: kept indices x*2^n + z
 *                (uint64, ascending) and their coefficients (c_type).  Only the
 *                first `cap` kept terms are written; cap = 0 (NULL outputs)
 *                just counts.
 *   d_count      device uint64: number of kept terms (may exceed cap).
 *   d_l1         device double: sum of |c_P| over every kept term.
 *   workspace    device, 256-byte aligned, ptdr_select_workspace_size() bytes.
 * The output order, count and normaliser are deterministic run to run.
 */
ptdr_status ptdr_coeff_select(int n, const void* C, ptdr_dtype c_type, double threshold,
                              unsigned long long k, uint64_t* d_idx, void* d_val, size_t cap,
                              unsigned long long* d_count, double* d_l1, void* workspace,
                              size_t workspace_bytes, void* stream);

/* Workspace bytes for ptdr_coeff_select.  Host only. */
ptdr_status ptdr_select_workspace_size(size_t* bytes);

/*
 * ptdr_probe_fp64_adds -- measurement helper, not part of the method (the
 * paper has no counterpart).  Enqueues an FP64 add-chain kernel of `blocks`
 * CTAs x `threads` threads, each running 8 independent chains of `iters`
 * dependent adds, and returns in *adds the number of FP64 adds it performs.
 * Timing it with events on `stream` gives the device's FP64 add rate, the
 * bound of the FP64 transforms.  d_sink: device scratch of `blocks` doubles
 * (never written in practice; it keeps the chains live).
 */
ptdr_status ptdr_probe_fp64_adds(void* d_sink, int blocks, int threads, int iters, double* adds,
                                 void* stream);

/* Human-readable name of a status code (static string, never NULL). */
const char* ptdr_status_string(ptdr_status status);

/* Library version, major * 10000 + minor * 100 + patch. */
int ptdr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PTDR_H */
