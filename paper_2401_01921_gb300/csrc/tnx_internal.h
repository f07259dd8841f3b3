// Internal declarations shared by the host planner and the CUDA kernels.
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include "tnx.h"

#define TNX_MAXR 8          // maximum rank of a tensor or an intermediate
#define TNX_MAXSYM 4        // maximum number of symmetries on a bond
#define TNX_QMAX (1 << 24)  // largest |charge| of a bond sector (sums over <= 8 legs stay inside int32)

// ---------------------------------------------------------------------------
// Device task descriptors (plain data, built on the host at plan time).
// A "slot" is an index into a device array of base pointers (double*), so a
// plan (and a CUDA graph captured from it) can be rebound to new input and
// output buffers by rewriting that array only.
// ---------------------------------------------------------------------------

// One strided block copy.  Legs are ordered outer -> inner; the last leg is
// the one contiguous in the destination.  src_slot < 0 writes zeros.
// Offsets inside one task are 32-bit (the planner rejects blocks whose
// element offsets reach 2^31); the slot offsets are 64-bit.  magic/shift
// divide an index below 2^31 by shape[l] without a hardware division:
// q = magic ? umulhi(n, magic) >> shift : n.
//
// Bands (tleg == TNX_BAND_HEADER): blocks that share the rows of one side's
// matrix ("wide" side: the packed GEMM operand they are written into, or the
// GEMM output they are read from), each covering a column range of those rows,
// move together in tiles staged through shared memory, so the wide side is
// accessed in whole rows and the other ("narrow") side along its own
// contiguous leg.  The header is followed by its `rank` members
// (tleg == TNX_BAND_MEMBER).  Header: wide slot in src_slot (source-wide) or
// dst_slot (destination-wide), the other slot -1; wide base offset in
// src_off / dst_off (element (p, q, c) of the band's rows lies at
// base + p * sstride[0] + q * sstride[1] + c); shape = {EP, EQ, W, TP, TQ,
// destination-wide, Q rows innermost in the tile}; nelem 0.  Member: rank 3
// with legs (P, Q, I) of extents (EP, EQ, n) and strides on both sides (the
// wide side's I stride is 1), wcol = its first column in the wide rows.
#define TNX_BAND_HEADER (-2)
#define TNX_BAND_MEMBER (-3)
struct CopyTask {
  int32_t src_slot, dst_slot;
  int32_t rank, tleg;         // tleg >= 0: transposing task, source contiguous along leg tleg; else -1 or a band mark
  int64_t src_off, dst_off;
  int64_t nelem;
  int32_t shape[TNX_MAXR];
  uint32_t magic[TNX_MAXR];
  int32_t sstride[TNX_MAXR];
  int32_t dstride[TNX_MAXR];
  uint8_t shift[TNX_MAXR];
  int32_t wcol, pad0;         // band member: first column in the wide rows
};

// One dense product C[M,N] = A[M,K] * B[N,K]^T (both operands K-major, C row-major).
struct GemmGroup {
  int32_t a_slot, b_slot, c_slot, pad0;
  int64_t a_off, b_off, c_off;
  int32_t M, N, K, lda, ldb, ldc;
};

struct GemmTile {
  int32_t group, m0, n0, pad0;
};

// Split-precision operand preparation: one packed FP64 matrix (rows x K,
// row-major, ld) is sliced into nslice integer-valued 16-bit slices written in
// the tcgen05 no-swizzle K-major core-matrix layout, tile by tile.
struct SliceJob {
  int32_t src_slot, dst_slot;     // dst: byte buffer slot (uint16 slices)
  int32_t exp_slot, wpg;          // int32 row exponents; warps per 8-row group (1, 2, 4 or 8)
  int64_t src_off, dst_off_bytes, exp_off;
  int32_t rows, K, ld, tile_rows; // tile_rows: 128 (A) or 64 (B)
  int32_t kx_slot, kx_sign;       // K balancing: int32 per K index (biased exponent of the
  int64_t kx_off;                 // column maximum of A), applied as 2^(kx_sign * E)
};

// K balancing of a split product: for every K index k of a charge group, the
// largest exponent field over the rows of the packed A (atomicMax into
// zeroed int32 words).  Items: (job, first K index, first row), 32 K indices
// by 64 rows each.
struct KexpJob {
  int32_t src_slot, kx_slot;
  int64_t src_off, kx_off;
  int32_t rows, K, ld, pad0;
};

// Split GEMM group: slices of A (tile_rows 128) and B (tile_rows 64) plus
// per-row / per-column exponents; output FP64 row-major.
struct SplitGroup {
  int32_t a_slot, b_slot, c_slot, ea_slot;
  int32_t eb_slot, out_slot, fc_slot, fc_off;   // fc_slot >= 0: the epilogue writes the network's output
  int64_t a_off_bytes, b_off_bytes, c_off, ea_off, eb_off;
  int32_t M, N, K, ldc;
};

// Output relayout folded into the last product's epilogue: column c of a
// charge group goes to out[off + r * stride] for its rows r (off < 0: the
// column is not part of the output).
struct FinalCol {
  int64_t off, stride;
};

// ---------------------------------------------------------------------------
// Fused charge-sector matching (integer): inputs of the device kernel.
// ---------------------------------------------------------------------------
struct MatchLeg {
  int32_t nsec;
  int32_t sec_base;     // offset into deg[] / charge[] arrays
};

struct MatchArgs {
  // legs
  int32_t nk, nfa, nfb, nsym;
  MatchLeg kleg[TNX_MAXR], faleg[TNX_MAXR], fbleg[TNX_MAXR];
  const int64_t* deg;        // degeneracies, indexed by sec_base + sector
  const int32_t* kcharge;    // signed charge of K-leg sectors as seen from A: [(sec_base+s)*nsym + c]
  int32_t zn[TNX_MAXSYM];    // 0 for U(1), n for Z_n
  int32_t clo[TNX_MAXSYM], crange[TNX_MAXSYM];
  // blocks
  int64_t nA, nB;
  int32_t rA, rB;
  const int32_t* qA;         // nA * rA sector indices (view leg order)
  const int32_t* qB;
  int32_t kposA[TNX_MAXR], fposA[TNX_MAXR], kposB[TNX_MAXR], fposB[TNX_MAXR];
  // sizes of the tuple spaces
  int64_t kspace, faspace, fbspace, cspace;
  // scratch (device)
  int32_t* kpres;  int32_t* kgroup;  int64_t* koff;
  int32_t* rgroup; int64_t* roff;
  int32_t* cgroup; int64_t* coff;
  int32_t* cspres; int32_t* csgid;
  int64_t* scan_tmp;        // 1024 * gmax
  int32_t gmax;
  // outputs (device)
  int32_t* ngroups;         // [1]
  int32_t* charges;         // gmax * nsym
  int64_t* mkn;             // gmax * 3
  int64_t* amap;            // nA * 3
  int64_t* bmap;            // nB * 3
  int32_t* status;          // [1]: 0 ok, 1 too many groups, 2 charge outside [clo, clo + crange),
                            //      3 a block's sector index outside its leg (nothing written)
};

// Counts kernel launches made by this library (defined in tnx_host.cpp).
// Programmatic dependent launch: every kernel of the library starts with
// tnx_grid_dependency(), which waits until the grids it depends on have
// completed and their writes are visible.  A kernel launched with tnx_launch
// may be launched as soon as every CTA of the previous kernel in the stream
// has exited (no explicit early trigger: waiting CTAs would take SM slots
// from the running kernel), so its launch overlaps the previous kernel's
// completion; without the launch attribute the wait returns at once.
#ifdef __CUDACC__
__device__ __forceinline__ void tnx_grid_dependency() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The skinny (MPO) products list the nonzero entries v of each output column
// of B and run acc = fma(a_k, v_k, acc) from acc = 0.  Their first term,
// fma(a, v, 0.0), is an exact scaling when v is a power of two (every MPO
// entry of the Heisenberg, XX and Hubbard chains is 0 or +-2^k), so it is
// formed on the integer units: flip the sign, add k to the exponent field.
// Zero, subnormal, infinite or out-of-range cases take the FMA; the result is
// bit-identical either way.  code = tnx_pow2_code(v): (sign << 31) | (biased
// exponent + 1), or 0 when v is not a normal power of two.
__host__ __device__ __forceinline__ uint32_t tnx_pow2_code(double v) {
  union {
    double d;
    unsigned long long u;
  } x;
  x.d = v;
  const unsigned ex = (unsigned)((x.u >> 52) & 0x7FF);
  if ((x.u & 0xFFFFFFFFFFFFFull) != 0 || ex == 0 || ex == 0x7FF) return 0u;
  return (unsigned)(x.u >> 63) << 31 | (ex + 1u);
}
__device__ __forceinline__ double tnx_first_term(double a, double v, uint32_t code) {
  if (code) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int ex = (int)((b >> 52) & 0x7FF);
    const int e = (int)(code & 0xFFFFu) - 1024;   // unbiased exponent of v
    if (ex > 0 && ex < 2047 && ex + e > 0 && ex + e < 2047)
      return __longlong_as_double((long long)((b ^ ((unsigned long long)(code >> 31) << 63)) +
                                              ((unsigned long long)(long long)e << 52)));
  }
  return fma(a, v, 0.0);
}

template <typename... KArgs, typename... Args>
cudaError_t tnx_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

void tnx_note_launch(long long n);   // kernel launches (into a graph's record while capturing)
void tnx_count_into(long long* c);    // nullptr: count globally again

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All enqueue on `st`.
// ---------------------------------------------------------------------------
cudaError_t tnx_launch_match(const MatchArgs& a, cudaStream_t st);
#define TNX_COPY_CHUNK 512     // elements per relayout CTA
#define TNX_COPY_PACK 64       // small tasks per relayout CTA at most
#define TNX_BAND_CAP 2048      // elements of a band tile staged in shared memory
#define TNX_BAND_MAXM 64       // members of a band at most
// chunks[i] = (first task, first element, task count, element count): a large
// task is cut into chunks of TNX_COPY_CHUNK elements (task count 1), runs of
// small tasks are packed (task count > 1, first element 0), a transposing
// task has one chunk per 32 x 32 tile: (task, tile index, -1, 0), and a band
// one chunk per tile: (header, tile index, -2, 0).
cudaError_t tnx_launch_copy(const CopyTask* tasks, const int4* chunks, int nchunks, double* const* slots,
                            cudaStream_t st);
// The same relayout (plain and transposing tasks only) reading src instead of
// each task's source slot, times *inv, plus vdst[i] = src[i] * *inv for
// i < vn (full != 0: the tasks read every such i exactly once and write it
// themselves); nothing is done when state[1] (a Lanczos stop flag) is set.
cudaError_t tnx_launch_copy_scaled(const CopyTask* tasks, const int4* chunks, int nchunks, double* const* slots,
                                   const double* src, double* vdst, int64_t vn, int full, const double* inv,
                                   const int32_t* state, cudaStream_t st);
// Fused skinny step (k_fused.cu): one CTA per tile of up to 128 rows (p, q),
// p in [p0, p0 + tP), q in [q0, q0 + tQ), of one row block of A_g (the rows a
// destination band of the step's relayout fills).  Column c < W (= ldK of the
// group) of those rows is described by FusedCol gcol + c: the A element of row
// (p, q) lies at ptr + p * sP + q * sQ (ptr null: a structural zero).  The rows
// are multiplied by the packed B_g (K <= 16, N <= 64) in FP64, and output
// column c < N of row (p, q) is stored through FusedCol scol + c the same way
// (ptr null: no step reads it).  scol < 0 writes the output rows to C_g
// instead: row (p, q) to row row0 + p * EQ + q of the group, EQ = -scol - 1.
// The pointers are plan buffers (fused steps read and write no rebindable
// slot).  kp, np: shared-memory pitches of the A and output rows (odd, > every
// W and N).
struct FusedCol {
  double* ptr;
  int32_t sP, sQ;
};
struct FusedTile {
  int32_t group, gcol, scol, row0;
  int32_t p0, q0, tP, tQ;
  int32_t W, N, pad0, pad1;
};
#define TNX_FUSED_ROWS 128   // rows (p, q) of a fused MPO-step tile at most (two threads per row)
cudaError_t tnx_launch_fused_skinny(const GemmGroup* groups, const FusedTile* tiles, int ntiles, const FusedCol* cols,
                                    int kp, int np, double* const* slots, cudaStream_t st);
size_t tnx_fused_smem_bytes(int kp, int np);
cudaError_t tnx_launch_gemm_f64(const GemmGroup* groups, const GemmTile* tiles, int ntiles,
                                double* const* slots, cudaStream_t st);
// K <= 16 products, tiles of 128 rows x 64 columns (FP64)
cudaError_t tnx_launch_gemm_skinny(const GemmGroup* groups, const GemmTile* tiles, int ntiles, double* const* slots,
                                   cudaStream_t st);
cudaError_t tnx_launch_gemm_f32(const GemmGroup* groups, const GemmTile* tiles, int ntiles,
                                double* const* slots, cudaStream_t st);
// row exponents, then the slices; items: (job, first 8-row group) per CTA work
// item, which covers 8 / wpg groups of that job
// Slicing straight from a Lanczos vector (the "vector mode" of the slicing
// kernel): row `row` of job j reads w + rowtab[j.src_off + row] (its K entries
// contiguous there), every entry is taken as w * (*inv), and that product is
// also written to vdst at the same offset (v_{j+1} = w / beta_{j+1}, the same
// FP64 product the normalising kernels form); nothing runs once state[1] (the
// Lanczos stop flag) is set.
struct VecSrc {
  const int64_t* rowtab;
  const double* w;
  double* vdst;
  const double* inv;
  const int32_t* state;
};
cudaError_t tnx_launch_slices_vec(const SliceJob* jobs, const int2* items, int64_t total_items, int nslice, int beta,
                                  int f16, double* const* slots, const VecSrc& vs, cudaStream_t st);
cudaError_t tnx_launch_slices(const SliceJob* jobs, const int2* items, int64_t total_items, int nslice, int beta,
                              int f16, double* const* slots, cudaStream_t st, int use_kx = 0);
// zero the K-balancing words of every job, then their column maxima
cudaError_t tnx_launch_kexp(const KexpJob* jobs, int njobs, const int4* items, int64_t nitems, double* const* slots,
                            cudaStream_t st);
// grid <= 0 or >= ntiles: one CTA per tile; otherwise a persistent grid of `grid` CTAs.
// tn: tile width (B rows per tile), 64 or 32; the B slices must be tiled with the same width.
cudaError_t tnx_launch_gemm_split(const SplitGroup* groups, const GemmTile* tiles, int ntiles, int nslice,
                                  int beta, int f16, double* const* slots, int32_t* status, cudaStream_t st,
                                  int grid, int tn, int mode = 0);   // mode: 0 plain, 1 folded output, 2 every K <= 160
size_t tnx_split_smem_bytes(int nslice, int tn);
// One-pass TF32 variant: tnx_launch_tf32_rows writes each operand row scaled by
// its power of two and rounded to TF32 (FP32 words, 16 K values per tile row,
// the same byte layout as one 16-bit slice); the GEMM runs kind::tf32 MMAs.
cudaError_t tnx_launch_tf32_rows(const SliceJob* jobs, const int2* items, int64_t total_items, double* const* slots,
                                 cudaStream_t st);
cudaError_t tnx_launch_gemm_tf32(const SplitGroup* groups, const GemmTile* tiles, int ntiles, double* const* slots,
                                 int32_t* status, cudaStream_t st, int grid, int tn, int fold = 0);

// ---------------------------------------------------------------------------
// SVD of dense charge blocks by one-sided Jacobi (k_svd.cu).  Per block: c
// working vectors of length r as the rows of X (c x r, row-major), the
// rotation accumulator J (c x c), sigma[c].
struct SvdGroup {
  double* X;
  double* J;
  double* sigma;
  int32_t c, r;
};
// One kept singular triplet: vector p of group g becomes column k of U (row
// stride ldu) and row k of V^T (row stride ldv); S (may be null) gets sigma at
// (k, k) with row stride lds.  absorb: 0 none, 1 sigma into V^T, 2 into U.
// cols_are_vectors: the working vectors are the columns of M (else its rows).
struct SvdOut {
  SvdGroup g;
  int32_t p, k, absorb, cols_are_vectors;
  double* U;
  double* Vt;
  double* S;
  int64_t ldu, ldv, lds;
};
// dst[i * dld + j] = src[i * sld + j] (trans: dst[j * dld + i]) for i < rows, j < cols
struct Copy2D {
  const double* src;
  double* dst;
  int64_t sld, dld;
  int32_t rows, cols, trans, pad0;
};
// The QR-preconditioned path of one block (k_svd.cu): A = X^T is r x c, its
// columns the working vectors.  The pivoted Householder QR A P = Q R runs in
// place in X; the one-sided Jacobi then works on the rows of R (Xr, with
// rotations Jr); Xf receives sigma_p u_p (u_p = Q Jr[p,:]^T, the left singular
// vectors of A) and J the right singular vectors of A as rows.
struct SvdQr {
  double* X;        // c x r
  double* tau;      // [c] reflector scalar of pivot position k
  int32_t* perm;    // [c] vector at pivot position k
  double* nrm;      // [2][c] squared norms of the trailing parts, by position
  int32_t* pos;     // [2][c] vector at each position
  double* Xr;       // c x c
  double* Jr;       // c x c
  double* Xf;       // c x r
  double* J;        // c x c
  double* sigma;    // [c]
  int32_t c, r;
};
cudaError_t tnx_launch_jacobi_init(const SvdGroup* groups, int ngroups, cudaStream_t st);
// the pivoted QR of every block in one cooperative launch over slots (block,
// position); *bar and *status zeroed by the caller; cudaErrorNotSupported
// without cooperative launch
cudaError_t tnx_launch_qr_coop(const SvdQr* qs, const int2* slots, int nslots, int maxc, unsigned long long* bar,
                               int* status, cudaStream_t st);
// Xr = R (rows, zero below the diagonal) and Jr = identity for every block
cudaError_t tnx_launch_qr_gather_r(const SvdQr* qs, int nq, int maxc, cudaStream_t st);
// after the Jacobi on Xr: sigma, J and Xf for every (block, vector)
// (maxr: the longest vector of the launch, which picks the register width)
cudaError_t tnx_launch_qr_apply(const SvdQr* qs, const int2* vecs, int nvec, int maxr, cudaStream_t st);
// round r of a sweep over slots (group, pair index); maxoff gets the largest
// |x_p . x_q| / (|x_p| |x_q|) met, as the bits of a non-negative double
// every round and sweep in one cooperative launch; offmax[max_sweeps], *bar
// and status zeroed by the caller; cudaErrorNotSupported without cooperative launch;
// maxlen: the longest vector or J row of the launch, which picks the register width
cudaError_t tnx_launch_jacobi_coop(const SvdGroup* groups, const int2* slots, int nslots, int maxcp, int maxlen,
                                   int max_sweeps, double tol, unsigned long long* offmax, unsigned long long* bar,
                                   int* status, int* sweeps_out, cudaStream_t st);
cudaError_t tnx_launch_jacobi_round(const SvdGroup* groups, const int2* slots, int nslots, int round,
                                    unsigned long long* maxoff, cudaStream_t st);
cudaError_t tnx_launch_vector_norms(const SvdGroup* groups, const int2* vecs, int nvec, cudaStream_t st);
cudaError_t tnx_launch_svd_extract(const SvdOut* outs, int nout, cudaStream_t st);
cudaError_t tnx_launch_copy2d(const Copy2D* tasks, int ntasks, cudaStream_t st);

// vector kernels (FP64, deterministic two-level reductions)
cudaError_t tnx_launch_scale(double* x, int64_t n, double alpha, cudaStream_t st);
cudaError_t tnx_launch_add_scalar(double* x, int64_t n, double alpha, cudaStream_t st);
cudaError_t tnx_launch_norm2(const double* x, int64_t n, double* partial, double* out, cudaStream_t st);
int tnx_reduce_blocks(int64_t n);

// Lanczos device state
struct LanczosDev {
  double* V;          // [nmax+1][n] basis
  double* w;          // [n]
  double* alpha;      // [nmax]
  double* beta;       // [nmax+1]
  double* coef;       // [nmax+1]  Gram-Schmidt coefficients
  double* partial;    // [nblocks * (nmax+1)]
  double* y;          // [nmax]    Ritz coefficients
  double* scratch;    // [4*nmax]
  int32_t* state;     // [0] = active steps done (k), [1] = stopped flag, [2] = this step reorthogonalises,
                      // [3] = the next step must reorthogonalise too, [4] = blocks done (last-block reductions)
  double* omega;      // [2][nmax+2] estimates of <v_j, v_k> (row j, then row j-1)
  double* eval;       // [1]
  int64_t n;
  int nmax;
  int nblocks;
};
cudaError_t tnx_launch_lanczos_init(const LanczosDev& L, const double* v0, cudaStream_t st);
cudaError_t tnx_launch_lanczos_set_input(double** slot_ptr, const LanczosDev& L, int j, cudaStream_t st);
// normalize = false leaves out v_{j+1} = w / beta_{j+1} (1 / beta_{j+1} is in
// scratch[3 * nmax + 3]) for the caller to fuse with its next relayout;
// always_pass: a Gram-Schmidt pass in every step (an operator far from symmetric)
cudaError_t tnx_launch_lanczos_step(const LanczosDev& L, int j, double** next_slot, cudaStream_t st, bool normalize,
                                    bool always_pass);
cudaError_t tnx_launch_lanczos_finish(const LanczosDev& L, double* evec, cudaStream_t st);
