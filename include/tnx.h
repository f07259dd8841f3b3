/*
 * tnx.h - C-ABI of the GB300 (sm_103a) block-sparse tensor-network library.
 *
 * The calls follow the problem statement of arXiv 2401.01921 ("The Cytnx
 * Library for Tensor Networks"): declare charged indices (bonds), build
 * block-sparse tensors, declare a network with its contraction order,
 * contract it, and run Lanczos on the contraction as a linear operator.
 * Section numbers below refer to that paper.
 *
 * Conventions shared by every call
 *  - All functions return a tnx_status: 0 (TNX_OK) or a negative error code.
 *    Nothing is thrown across the ABI.  tnx_last_error(ctx) returns a
 *    NUL-terminated message for the last failing call made with that context
 *    (thread-unsafe: one context per host thread).
 *  - Device memory comes from the allocator callback given to
 *    tnx_ctx_create (NULL callbacks: cudaMallocAsync / cudaFreeAsync on the
 *    context stream).  The library never frees memory it did not allocate.
 *  - Work is enqueued asynchronously on the context stream; tnx_sync and the
 *    blocking getters (tnx_tensor_get_block, tnx_lanczos results) join it.
 *  - Element type: FP64 (double) everywhere on the public surface.
 *  - Handles are owned by the caller, who destroys each one exactly once.
 *    A network keeps references to the tensors put into it (no copy, the
 *    reference semantics of Sec. 3.2); a tensor must outlive its use by a
 *    network launch.
 */
#ifndef TNX_H
#define TNX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tnx_status;

enum {
  TNX_OK = 0,
  TNX_ERR_ARG = -1,            /* invalid argument, NULL handle, out-of-range size */
  TNX_ERR_BOND_MISMATCH = -2,  /* contracted bonds differ in dimension, direction,
                                  charges or block dimensions (Sec. 7) */
  TNX_ERR_SYMMETRY = -3,       /* operation would break the block structure: scalar
                                  add on a symmetric tensor (Sec. 6.3), symmetry-
                                  violating entry in a conversion (Sec. 6.5) */
  TNX_ERR_NO_BLOCK = -4,       /* the requested block does not exist (Sec. 6.3.2) */
  TNX_ERR_NETWORK = -5,        /* network text, missing put, bad ORDER (Sec. 8) */
  TNX_ERR_OOM = -6,            /* allocator returned NULL */
  TNX_ERR_TIMEOUT = -7,        /* a bounded device wait ran out */
  TNX_ERR_CUDA = -8,           /* a CUDA runtime call failed */
  TNX_ERR_UNSUPPORTED = -9     /* shape outside the implemented limits */
};

/* Symmetry kinds (Sec. 6.1): U(1) combines by addition; Z_n by (Q1+Q2) mod n.
 * Both reverse a charge by negation (mod n for Z_n). */
enum { TNX_U1 = 0, TNX_ZN = 1 };

/* Bond directions (Sec. 4, Sec. 6.2): IN (ket) = +1, OUT (bra) = -1,
 * REGULAR (no symmetry) = 0. */
enum { TNX_BD_IN = 1, TNX_BD_OUT = -1, TNX_BD_REG = 0 };

/* Arithmetic of the block products (not part of the paper; the paper's GPU
 * path uses library FP64 GEMMs, Sec. 10).
 *  TNX_PREC_F64       native FP64 products.
 *  TNX_PREC_SPLIT_BF16 / _F16  error-free slicing of each FP64 operand into
 *      integer-valued BF16 / FP16 slices with a common power-of-two scale per
 *      row of A and per column of B (Ozaki, Ogita, Oishi, Rump, "Error-free
 *      transformations of matrix multiplication by using fast routines of
 *      matrix multiplication and its applications", Numer. Algorithms 59,
 *      2012); slice products on the tcgen05 tensor cores, exact in FP32 over
 *      K chunks, recombined exactly in 64-bit integers, rounded once to FP64.
 *  TNX_PREC_F32       operands rounded to FP32, FP32 products and sums.
 *  TNX_PREC_TF32      one pass on the tcgen05 tensor cores (kind::tf32): each
 *      row of A / column of B scaled by a power of two and rounded to TF32
 *      (11 significant bits, nearest-even), FP32 sums over 640-long K chunks,
 *      chunks summed in FP64.  Relative error about 2^-11 of the products.
 *  In every variant, charge groups whose K is at most 16 (the MPO products)
 *  run as FP64 products. */
enum { TNX_PREC_F64 = 0, TNX_PREC_SPLIT_BF16 = 1, TNX_PREC_SPLIT_F16 = 2,
       TNX_PREC_F32 = 3, TNX_PREC_TF32 = 4 };

typedef struct tnx_ctx tnx_ctx;
typedef struct tnx_bond tnx_bond;
typedef struct tnx_tensor tnx_tensor;
typedef struct tnx_network tnx_network;

/* Device allocator callback: returns a device pointer of at least nbytes
 * (256-byte aligned) or NULL.  free receives exactly the pointers alloc
 * returned.  Both are called on the host thread that makes the tnx call. */
typedef void* (*tnx_alloc_fn)(size_t nbytes, void* user);
typedef void (*tnx_free_fn)(void* ptr, size_t nbytes, void* user);

/* ---------------------------------------------------------------- context */

/* Returns the message of the last error on ctx (never NULL). */
const char* tnx_last_error(const tnx_ctx* ctx);

/* Library version string ("tnx <major>.<minor>"). */
const char* tnx_version(void);

/* Create a context on CUDA device `device`, enqueueing on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  alloc/free may be NULL
 * (stream-ordered CUDA allocation).  *out receives the handle. */
tnx_status tnx_ctx_create(int device, void* stream, tnx_alloc_fn alloc, tnx_free_fn free,
                          void* alloc_user, tnx_ctx** out);
/* Destroys the context; tensors, bonds and networks made with it must be
 * destroyed first.  Synchronises the stream. */
tnx_status tnx_ctx_destroy(tnx_ctx* ctx);
/* Blocks until all work enqueued on the context stream has finished. */
tnx_status tnx_sync(tnx_ctx* ctx);

/* ------------------------------------------------------------------ bonds */

/* A bond with quantum numbers (Sec. 6.2.1): direction, nsym symmetries
 * (kinds[i] in {TNX_U1, TNX_ZN}, zn[i] = n for Z_n, ignored for U(1)), and nsec
 * sectors in creation order, sector k having charges qnums[k*nsym .. k*nsym+nsym)
 * and degeneracy degs[k] >= 1.  nsym = 0 with dir = TNX_BD_REG makes a plain
 * bond of dimension degs[0] (nsec must be 1).  Arrays are copied.  Charges
 * beyond |q| = 2^24 and Z_n moduli above 2^24 give TNX_ERR_UNSUPPORTED (also
 * for tnx_bond_combine results). */
tnx_status tnx_bond_create(tnx_ctx* ctx, int dir, int nsym, const int* kinds, const int* zn,
                           int nsec, const int32_t* qnums, const int64_t* degs, tnx_bond** out);
/* Total dimension (sum of degeneracies). */
tnx_status tnx_bond_dim(const tnx_bond* b, int64_t* dim);
/* Sec. 6.2.2: combine two bonds with equal direction and symmetries; sectors
 * with equal charge are grouped, the result is sorted ascending by charge. */
tnx_status tnx_bond_combine(const tnx_bond* a, const tnx_bond* b, tnx_bond** out);
/* Number of sectors, and (optional, may be NULL) their charges and degeneracies. */
tnx_status tnx_bond_sectors(const tnx_bond* b, int* nsec, int32_t* qnums, int64_t* degs);
/* Direction and symmetries (any pointer may be NULL; kinds / zn hold nsym entries). */
tnx_status tnx_bond_info(const tnx_bond* b, int* dir, int* nsym, int* kinds, int* zn);
tnx_status tnx_bond_destroy(tnx_bond* b);

/* ---------------------------------------------------------------- tensors */

/* Sec. 6.3.1: a block-sparse FP64 tensor over `rank` bonds (copied).  Only
 * zero-flux blocks are stored: the charges of IN legs combined with the
 * reversed charges of OUT legs vanish.  Blocks are numbered in lexicographic
 * order of their sector indices ("Qn indices"); each block is a dense
 * row-major array over the tensor's leg order; the blocks lie back to back in
 * one device buffer, zero-filled.  rank = 0 gives a scalar (one element). */
tnx_status tnx_tensor_create(tnx_ctx* ctx, int rank, tnx_bond* const* bonds, tnx_tensor** out);
tnx_status tnx_tensor_destroy(tnx_tensor* t);
tnx_status tnx_tensor_rank(const tnx_tensor* t, int* rank);
tnx_status tnx_tensor_nblocks(const tnx_tensor* t, int64_t* n);
/* Block `blk`: its sector indices qn_idx[rank], shape[rank] and element offset
 * in the buffer (any output pointer may be NULL). */
tnx_status tnx_tensor_block_info(const tnx_tensor* t, int64_t blk, int32_t* qn_idx, int64_t* shape,
                                 int64_t* offset);
/* All blocks at once: qn_idx[nblk*rank], shape[nblk*rank], offset[nblk] (any may be NULL). */
tnx_status tnx_tensor_blocks(const tnx_tensor* t, int32_t* qn_idx, int64_t* shape, int64_t* offset);
/* A new bond handle (caller owns) equal to leg `leg` of t. */
tnx_status tnx_tensor_bond(const tnx_tensor* t, int leg, tnx_bond** out);
/* Borrowed device pointer to the element buffer and its element count. */
tnx_status tnx_tensor_data(tnx_tensor* t, double** dev_ptr, int64_t* nelem);
/* Copy host data into the block with sector indices qn_idx (n = its size);
 * TNX_ERR_NO_BLOCK if that block is not stored (Sec. 6.3.2). Synchronous. */
tnx_status tnx_tensor_put_block(tnx_tensor* t, const int32_t* qn_idx, const double* host, int64_t n);
/* Copy the block out to host memory.  Synchronous. */
tnx_status tnx_tensor_get_block(const tnx_tensor* t, const int32_t* qn_idx, double* host, int64_t n);
/* Whole buffer host <-> device (n = nelem), synchronous. */
tnx_status tnx_tensor_upload(tnx_tensor* t, const double* host, int64_t n);
tnx_status tnx_tensor_download(const tnx_tensor* t, double* host, int64_t n);
/* Sec. 6.3: multiply / divide by a scalar is allowed (t *= alpha). */
tnx_status tnx_tensor_scale(tnx_tensor* t, double alpha);
/* Sec. 6.3: adding a scalar would break the block structure; always returns
 * TNX_ERR_SYMMETRY for a tensor with symmetric bonds (plain tensors: t += alpha). */
tnx_status tnx_tensor_add_scalar(tnx_tensor* t, double alpha);
/* Two-norm over the stored elements (FP64, device reduction).  Synchronous. */
tnx_status tnx_tensor_norm(const tnx_tensor* t, double* out);
/* Sec. 6.4 Dagger: a new tensor (caller owns) with every bond redirected
 * (IN <-> OUT; REGULAR bonds stay) and the same blocks and data (the elements
 * are real, so complex conjugation changes nothing).  Asynchronous copy on
 * the context stream. */
tnx_status tnx_tensor_dagger(const tnx_tensor* t, tnx_tensor** out);

/* ---------------------------------------------------------- decomposition */

/* Sec. 9.1 / 9.2 Svd and Svd_truncate of a block-sparse tensor.  The first
 * `rowrank` legs are the row legs (1 <= rowrank < rank); the matrix form has
 * one dense block per total charge g of the row legs (blocks of S in
 * ascending order of g).  Every block gets a full SVD on the device (one-sided
 * Jacobi, FP64); then the singular values of all blocks are sorted together
 * and the largest keepdim are kept (keepdim <= 0: no limit), values below err
 * are dropped (err <= 0: none; values are not normalised), and
 * min_blockdim[i] (nmin = number of blocks of S, or min_blockdim = NULL)
 * values of block i are kept even if the other rules drop them; those count
 * towards keepdim.  Equal values are ranked by block, then position.
 * Outputs (new tensors, caller owns): U with the row legs and a new OUT leg
 * whose sectors are the kept charges (ascending) with the kept counts; S, a
 * diagonal [IN, OUT] tensor over the new leg (may be NULL unless absorb == 0);
 * Vdag with the new IN leg followed by the column legs.  absorb = 1 returns
 * S * Vdag in Vdag, absorb = 2 returns U * S in U.  trunc_err (may be NULL):
 * the largest dropped value (0 if none), as return_err = 1; discarded (may be
 * NULL): the sum of the dropped values squared.  Plain (REGULAR) tensors give
 * a REGULAR new leg.  TNX_ERR_ARG if nothing is kept or the arguments are
 * inconsistent.  Synchronous. */
tnx_status tnx_svd_truncate(tnx_tensor* t, int rowrank, int64_t keepdim, double err, const int64_t* min_blockdim,
                            int nmin, int absorb, tnx_tensor** U, tnx_tensor** S, tnx_tensor** Vdag,
                            double* trunc_err, double* discarded);

/* --------------------------------------------------------------- networks */

/* Sec. 8.1: a network blueprint from text, one entry per line:
 *   "NAME: l1, l2, ..."   a tensor and its dummy labels (labels on two
 *                         tensors are summed over; hyperedges and traces
 *                         are rejected),
 *   "TOUT: l1, l2; l3"    the open labels in output order (';' accepted as a
 *                         separator; empty = scalar output),
 *   "ORDER: ((A,B),C)"    optional contraction tree; empty = order of
 *                         appearance.
 * Errors: TNX_ERR_NETWORK. */
tnx_status tnx_network_create(tnx_ctx* ctx, const char* spec, tnx_network** out);
tnx_status tnx_network_destroy(tnx_network* net);
/* Sec. 8.2 PutUniTensor: labels[i] is the blueprint label that leg i of `t`
 * realises (nlab == rank; labels == NULL: t's legs follow the blueprint line).
 * The network keeps a reference to t.  Bond checks happen at launch. */
tnx_status tnx_network_put(tnx_network* net, const char* name, tnx_tensor* t, int nlab,
                           const char* const* labels);
/* Sec. 8.3 setOrder: optimal == 1 computes the min-cost order (dynamic
 * programming with cost capping, Pfeifer et al. 2014, cost = product of the
 * dimensions of all legs of each pairwise contraction) at launch, cached per
 * set of bond dimensions; optimal == 0 takes `order` ("(A,(B,C))").
 * optimal == 2 (an addition to the paper's search, for block-sparse
 * operands): the same subset dynamic programming with each pairwise cost
 * counted over charge sectors, 2 * sum_g H_a(-g) H_k(g) H_b(g), H_S(c) = number
 * of index combinations of the legs S with signed total charge c, assuming
 * every intermediate holds all zero-flux blocks of its legs; at most 12
 * tensors (else TNX_ERR_UNSUPPORTED); cached per set of bond sectors.
 * Errors: TNX_ERR_ARG (optimal outside 0..2), TNX_ERR_NETWORK. */
tnx_status tnx_network_set_order(tnx_network* net, int optimal, const char* order);
/* Sec. 8.3 getOrder: writes the current tree ("(M2,(M1,M3))"), NUL-terminated,
 * into buf (TNX_ERR_ARG if len is too small). */
tnx_status tnx_network_get_order(const tnx_network* net, char* buf, size_t len);
/* Arithmetic of the block products (TNX_PREC_*); default TNX_PREC_F64. */
tnx_status tnx_network_set_precision(tnx_network* net, int prec);
/* Sec. 8.2 Launch: contract all tensors; returns a new tensor (caller owns)
 * with the TOUT legs, every zero-flux block stored.  Asynchronous. */
tnx_status tnx_network_launch(tnx_network* net, tnx_tensor** out);
/* Launch into a preallocated tensor whose bonds equal the TOUT bonds. */
tnx_status tnx_network_launch_into(tnx_network* net, tnx_tensor* out);
/* Useful flops of one launch at the current order: 2*m*k*n summed over the
 * matched block pairs of every pairwise contraction (plans if needed). */
tnx_status tnx_network_flops(tnx_network* net, double* flops);
/* Device bytes the network holds now (plan buffers and Lanczos workspace);
 * *plan_bytes (may be NULL) gets the bytes its plan needs at the current
 * order and bonds, sized without allocating when no plan is built. */
tnx_status tnx_network_resident(tnx_network* net, size_t* bytes, size_t* plan_bytes);
/* Number of pairwise contractions in the plan (= number of tensors - 1). */
tnx_status tnx_network_nsteps(tnx_network* net, int* nsteps);
/* Fused charge-sector tables of pairwise contraction `step` (post-order of the
 * tree), as built by the device matching kernel.  Sizes first: ngroups,
 * nsym, and the block counts of the two operands.  Then the tables (any
 * pointer may be NULL): charges[ngroups*nsym] (ascending), mkn[ngroups*3]
 * (M, K, N), amap[nA*3] (group, row offset, K offset; -1 if unused),
 * bmap[nB*3] (group, K offset, column offset).  Operand blocks are listed in
 * lexicographic order of their sector indices in blueprint leg order. */
tnx_status tnx_network_step_sizes(tnx_network* net, int step, int* ngroups, int* nsym, int64_t* nA,
                                  int64_t* nB);
tnx_status tnx_network_step_tables(tnx_network* net, int step, int32_t* charges, int64_t* mkn,
                                   int64_t* amap, int64_t* bmap);

/* ---------------------------------------------------------------- Lanczos */

/* Sec. 9.3 Lanczos on a LinOp: the network, with the tensor named `vec_slot`
 * as the vector, is the linear operator (its TOUT bonds must equal the
 * vector's bonds), which must be Hermitian.  Starting from v0, runs at most
 * nsteps Lanczos steps (three-term recurrence) that keep the basis orthogonal
 * to 1e-10 or better: each step estimates the loss of orthogonality by
 * Simon's recurrence (partial reorthogonalisation) and takes a classical
 * Gram-Schmidt pass against all earlier vectors when an estimate exceeds
 * 1e-10 (and at the next step too); in TNX_PREC_F32 and TNX_PREC_TF32, whose
 * rounded operator is far from symmetric, every step takes the pass.  Stops
 * early if the new off-diagonal falls below 1e-14 * max(|alpha_i|, beta_i) over
 * the steps so far; returns the lowest
 * eigenvalue of the tridiagonal matrix (Sturm bisection, FP64) in *eval and,
 * if evec != NULL, the Ritz vector (unit norm, largest-|y| coefficient
 * positive) in evec (same bonds as v0).  *nmatvec (may be NULL) gets the number
 * of operator applications.  All vector arithmetic runs in FP64 on the device;
 * the apply uses the network's precision.  Synchronous. */
tnx_status tnx_lanczos(tnx_network* net, const char* vec_slot, tnx_tensor* v0, int nsteps,
                       double* eval, tnx_tensor* evec, int* nmatvec);

/* ------------------------------------------------------------------- DMRG */

/* The two-site DMRG sweep of Sec. 11 (the benchmark around Fig. "Hpsi_fig"),
 * built from the calls above: per bond, the two-site wavefunction A_i A_{i+1}
 * (a network launch), its lowest eigenvector under H_eff = (L, W, W, R) by
 * tnx_lanczos, the split by tnx_svd_truncate (S absorbed towards the sweep
 * direction), and the environment update L.A.W.A^dagger or A.W.R.A^dagger (a
 * network launch).  W is the uniform MPO [wL IN, s' IN, s OUT, wR OUT] (copied;
 * REGULAR legs for a plain chain); left_w / right_w are the dense MPO indices
 * the chain's left / right edges select; states[nsites] is the initial product
 * state (dense indices into the physical leg), which also fixes the total
 * charge.  MPS tensors are A_i[a IN, s IN, b OUT].  No counterpart as a call in
 * the paper (its sweep is a user-guide example). */
typedef struct tnx_dmrg tnx_dmrg;
tnx_status tnx_dmrg_create(tnx_ctx* ctx, int nsites, const tnx_tensor* W, int left_w, int right_w,
                           const int32_t* states, tnx_dmrg** out);
tnx_status tnx_dmrg_destroy(tnx_dmrg* d);
/* One sweep (left to right, then right to left) keeping at most maxdim values
 * per bond and dropping values below cutoff, lanczos_steps steps per update,
 * H_eff products in precision prec (TNX_PREC_*).  Outputs (any may be NULL):
 * the last Lanczos eigenvalue, the largest dropped singular value, the largest
 * bond dimension, and host milliseconds per phase [two-site wavefunction and
 * Lanczos, SVD, environments, whole sweep].  Synchronous. */
tnx_status tnx_dmrg_sweep(tnx_dmrg* d, int64_t maxdim, double cutoff, int lanczos_steps, int prec, double* energy,
                          double* max_trunc_err, int64_t* max_bond, double* phase_ms);
/* A copy of the MPS tensor of site `site` (caller owns). */
tnx_status tnx_dmrg_tensor(const tnx_dmrg* d, int site, tnx_tensor** out);

/* ---------------------------------------------------------------- batches */

/* A batch of nnet networks with the same number of pairwise contractions and
 * the same precision (typically one blueprint over many independent
 * instances: the batched H_eff*psi of many DMRG problems).  Every pairwise
 * step of all instances runs as one relayout launch and one grouped-GEMM
 * launch over all their charge sectors; a launch of the batch is one CUDA
 * graph.  Each network must be fully put; its plan is built now and the batch
 * keeps references (a network must outlive the batch; re-planning a network
 * invalidates the batch: TNX_ERR_ARG at launch).  A network that joins a batch
 * keeps 64-wide split-GEMM tiles from then on (one merged launch needs one tile
 * width).  No counterpart in the paper, which contracts one network per call
 * (Sec. 8). */
typedef struct tnx_batch tnx_batch;
tnx_status tnx_batch_create(tnx_ctx* ctx, int nnet, tnx_network* const* nets, tnx_batch** out);
tnx_status tnx_batch_destroy(tnx_batch* b);
/* Launch every network into outs[i] (bonds equal to network i's TOUT bonds). Asynchronous. */
tnx_status tnx_batch_launch_into(tnx_batch* b, tnx_tensor* const* outs);
/* Useful flops of one batch launch (sum over the instances). */
tnx_status tnx_batch_flops(tnx_batch* b, double* flops);
/* Times the split-GEMM launch schedules (one CTA per tile; persistent grids of
 * 152, 304, 456 CTAs) on this batch (writing into outs) and keeps the fastest;
 * *choice (may be NULL) gets the grid size (0 = one CTA per tile). */
tnx_status tnx_batch_autotune(tnx_batch* b, tnx_tensor* const* outs, int* choice);

/* ---------------------------------------------------------------- serving */

/* A serving loop with continuous batching (no counterpart in the paper).  A
 * request is one H_eff*psi-style apply (TNX_REQ_APPLY: out = the network
 * applied with `vec` in slot `vec_slot`) or a Lanczos solve (TNX_REQ_LANCZOS:
 * nsteps steps from `vec`; out, optional, receives the Ritz vector).  The
 * networks stay resident (plans, packed constant operands, Lanczos workspace)
 * between requests.  A worker thread admits queued requests, first fit in
 * arrival order, whenever one of max_slots stream slots is free, the request's
 * network is idle (one request per network at a time) and its resident memory
 * fits hbm_budget_bytes (idle networks are evicted least recently used first);
 * admitted requests run concurrently on their own CUDA streams.  While a
 * server runs, the networks it serves must not be launched or modified through
 * other calls, and the context's allocator must be callable from the worker
 * thread. */
enum { TNX_REQ_APPLY = 0, TNX_REQ_LANCZOS = 1 };
typedef struct tnx_server tnx_server;
tnx_status tnx_server_create(tnx_ctx* ctx, int max_slots, size_t hbm_budget_bytes, tnx_server** out);
/* Stops the worker (requests not yet started are dropped), waits for running ones. */
tnx_status tnx_server_destroy(tnx_server* s);
/* Queues a request; *id identifies it for tnx_server_wait.  Thread-safe. */
tnx_status tnx_server_submit(tnx_server* s, tnx_network* net, const char* vec_slot, tnx_tensor* vec, int kind,
                             int nsteps, tnx_tensor* out, int64_t* id);
/* Blocks until request id finishes (timeout_ms < 0: no limit; TNX_ERR_TIMEOUT
 * if it runs out) and returns its status; eval / matvecs (Lanczos) and the
 * latency from submission to completion in milliseconds (any may be NULL).
 * Each id can be waited for once. */
tnx_status tnx_server_wait(tnx_server* s, int64_t id, int timeout_ms, double* eval, int* matvecs, double* latency_ms);
/* Completed requests, evictions, bytes currently resident, peak resident bytes. */
tnx_status tnx_server_stats(tnx_server* s, int64_t* completed, int64_t* evictions, size_t* used_bytes,
                            size_t* peak_bytes);

/* ------------------------------------------------- no-allocation variant */

/* The fused charge-sector tables of ONE pairwise contraction (what
 * tnx_network_step_tables reports for a step), computed by the device matching
 * kernel WITHOUT allocating any memory.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc (or any allocator) where they need
 * the tables - a latency-critical loop whose memory was sized up front, a
 * process whose device memory belongs to another framework's pool, a plugin
 * that only receives pre-sized buffers.  No tnx_ctx is needed (creating one
 * allocates).
 *
 * The kernel's working memory is a fixed 16 MiB array in device memory that
 * every GPU loading the library holds until the process exits; contractions
 * that need more are refused (TNX_ERR_UNSUPPORTED, with the byte count in err).
 * Every call shares that array: calls that overlap on the GPU race and must be
 * serialised by the caller.  The first call on a device looks up the array's
 * device address (with that device current); make that first call before any
 * stream capture.  The call enqueues on `stream` (a cudaStream_t, NULL = legacy
 * default stream) and waits for it before returning.
 *
 * Arguments (host = host memory, dev = device memory):
 *  nsym, zn[nsym] (host): symmetries; zn[c] = 0 for U(1), n for Z_n.
 *  nk, nfa, nfb: contracted legs, free legs of A, free legs of B.
 *  nsec[nk+nfa+nfb] (host): sectors per leg, K legs (in A's leg order) first.
 *  degs (host): degeneracies of every sector of those legs, concatenated.
 *  kcharges (host): [K-leg sector][nsym] charges as they enter A's flux
 *      (negated on OUT legs, reduced mod n for Z_n).
 *  nA, rA, qA (dev, int32 [nA*rA]): A's blocks (sector indices, lexicographic);
 *      the kernel checks every entry against its leg's sector count before it
 *      writes anything and returns TNX_ERR_ARG (no table written) if one is
 *      out of range;
 *  kposA[nk], fposA[nfa] (host): A's legs holding the K / free legs; together
 *      they must name each of A's rA legs exactly once (TNX_ERR_ARG otherwise);
 *      same for B.
 *  Limits (TNX_ERR_UNSUPPORTED beyond them): sector tuple spaces and the charge
 *      space of the K legs at most 2^24 entries, |charge| <= 2^24, Z_n moduli
 *      at most 2^22.
 *  gmax: capacity of the group outputs.
 *  Outputs (dev): ngroups[1], charges[gmax*nsym], mkn[gmax*3],
 *      amap[nA*3], bmap[nB*3] - the same conventions as tnx_network_step_tables.
 *  err[errlen] (host, may be NULL): message on failure, empty on success. */
tnx_status tnx_match_tables_noalloc(void* stream, int nsym, const int32_t* zn, int nk, int nfa, int nfb,
                                    const int32_t* nsec, const int64_t* degs, const int32_t* kcharges,
                                    int64_t nA, int rA, const int32_t* qA, const int32_t* kposA,
                                    const int32_t* fposA, int64_t nB, int rB, const int32_t* qB,
                                    const int32_t* kposB, const int32_t* fposB, int gmax, int32_t* ngroups,
                                    int32_t* charges, int64_t* mkn, int64_t* amap, int64_t* bmap, char* err,
                                    size_t errlen);

/* ------------------------------------------------------------ diagnostics */

/* Kernel classes timed by the profiler. */
enum { TNX_KC_MATCH = 0, TNX_KC_RELAYOUT = 1, TNX_KC_GEMM = 2, TNX_KC_SLICE = 3, TNX_KC_VECTOR = 4,
       TNX_KC_FINAL = 5, TNX_KC_SKINNY = 6, TNX_KC_COUNT = 7 };

/* enable != 0: bracket every kernel class a launch enqueues on the context
 * stream with CUDA events (adds two event records per launch); 0 stops.
 * Resets the accumulated figures either way. */
tnx_status tnx_profile_enable(tnx_ctx* ctx, int enable);
/* As tnx_profile_enable, for the classes whose bit (1 << TNX_KC_*) is set in
 * class_mask only (0 stops): the event records of the other classes are left
 * out of the stream and of captured graphs.  With TNX_PROF_LAST_APPLY also
 * set, a Lanczos solve times only the operator apply of its last step (event
 * records in a captured graph cost time of their own; a solve's applies run
 * the same kernels on the same shapes). */
#define TNX_PROF_LAST_APPLY 0x80000000u
tnx_status tnx_profile_classes(tnx_ctx* ctx, uint32_t class_mask);
/* Synchronises the stream and returns, per kernel class (arrays of
 * TNX_KC_COUNT entries, any may be NULL): summed device milliseconds, number
 * of launches, and the algorithmic work of those launches (useful flops for
 * TNX_KC_GEMM (the main grouped product: split tensor-core or FP64) and
 * TNX_KC_SKINNY (the K <= 16 FP64 products): 2*m*k*n over matched block pairs;
 * bytes read + written for the relayout and slice classes, each element counted
 * once per direction). */
tnx_status tnx_profile_read(tnx_ctx* ctx, double* ms, int64_t* launches, double* work);
/* Number of CUDA kernels this library has launched in the process so far. */
tnx_status tnx_kernel_launches(int64_t* n);

#ifdef __cplusplus
}
#endif
#endif /* TNX_H */
