/*
 * spand.h -- C ABI of the GB300 spaND (sparsified nested dissection) library.
 *
 * Problem (Sec. 1, Eq. (1)): solve A x = b for a sparse symmetric
 * positive-definite A in R^{N x N}.  The only required input is A; vertex
 * coordinates are optional and, when given, drive the geometric vertex
 * separator (Sec. 2.3, last paragraph).  The library
 *   1. analyzes A on the host: modified nested-dissection ordering and
 *      clustering (Algorithm 3, Sec. 2.3) plus the symbolic structure of every
 *      elimination step (fill, Sec. 2.4; merge maps, Sec. 2.7; colouring of
 *      the sparsification order);
 *   2. factorizes on the GPU, level by level (Algorithm 2, "OrthS"): block
 *      Cholesky elimination of every separator (Sec. 2.4), block-diagonal
 *      scaling of every interface (Sec. 2.5), orthogonal sparsification by
 *      column-pivoted QR truncated at eps (Sec. 2.6.1; truncation rule of
 *      Sec. 4), merge (Sec. 2.7), giving M with M^T A M ~ I (Sec. 2.8);
 *   3. solves with preconditioned CG on the GPU, the preconditioner being
 *      z = M M^T r (Sec. 2.8), to ||b - A x||_2 / ||b||_2 <= tol (Sec. 4).
 *
 * Conventions for every call:
 *   - Return value: SPAND_OK (0) or one of the SPAND_ERR_* codes below; no C++
 *     exception crosses this boundary.  spand_last_error() gives a message.
 *   - The caller owns every array it passes; the library copies what it keeps.
 *   - CSR: rowptr int64[n+1] (rowptr[0] = 0), colind int32[nnz] strictly
 *     increasing within each row, every diagonal entry present, symmetric
 *     pattern; vals float64[nnz] of a symmetric matrix.
 *   - Pointers are host pointers unless a call says otherwise.  Vector
 *     arguments of spand_solve may be host or device memory (detected with
 *     cudaPointerGetAttributes).
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Every
 *     call that takes a stream returns after its work on that stream is done.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef SPAND_H
#define SPAND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SPAND_OK = 0,
  SPAND_ERR_INVALID_ARG = 1,   /* bad size, null pointer, malformed CSR */
  SPAND_ERR_NOT_SPD = 2,       /* a pivot block is not positive definite */
  SPAND_ERR_NO_CONVERGENCE = 3,/* PCG reached maxit above tol */
  SPAND_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  SPAND_ERR_OOM = 5,           /* device or host allocation failed */
  SPAND_ERR_STATE = 6,         /* call out of order (e.g. solve before factorize) */
  SPAND_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up (the context
                                  stays usable; the call's result is invalid) */
};

/* precision of the factorization (the PCG recurrences, its dot products
 * and the SpMV always run in FP64, and so does the Cholesky of every pivot
 * block: the eliminated separators of Sec. 2.4 and the scaled interfaces of
 * Sec. 2.5) */
enum {
  SPAND_FP64 = 0,  /* plain: every factor kernel in FP64 */
  SPAND_FP32 = 1,  /* mixed: factor stored in FP32; pivot and scaling Cholesky
                      in FP64 (on an FP64 copy of each pivot block, U and the
                      inverses of its diagonal tiles rounded to FP32);
                      triangular solves, Schur GEMMs, QR and the
                      preconditioner apply in FP32; vectors, SpMV and the PCG
                      recurrences in FP64 */
  SPAND_TF32 = 2,  /* as SPAND_FP32, with the elimination's Schur GEMMs on the
                      tensor cores: TF32 operands, FP32 accumulation */
  SPAND_BF16 = 3   /* as SPAND_TF32 with BF16 operands (FP32 accumulation,
                      factor stored in FP32) */
};

/* order of the sparsifications inside a level (Algorithm 2 applies S_p to
 * every interface p of the level; Sec. 2.6.1) */
enum {
  SPAND_COLOURED = 0,     /* greedy distance-1 colouring of the interfaces;
                             colours in sequence, each interface compressed
                             from the matrix its earlier-coloured neighbours
                             left (a sequential order of Algorithm 2) */
  SPAND_SIMULTANEOUS = 1  /* every interface compressed from the same scaled
                             matrix, then every coupling block transformed
                             from both sides, A_pq <- Q_pc^T A_pq Q_qc (one
                             launch per level; the kept matrix is a principal
                             submatrix of an orthogonal similarity, so SPD);
                             differs from the coloured order at O(eps) */
};

/* how each interface is compressed (Sec. 2.6) */
enum {
  SPAND_CPQR = 0,       /* column-pivoted QR of A_pn truncated at eps (Sec. 2.6.1, rule of Sec. 4) */
  SPAND_RANDOMIZED = 1  /* randomized range finder (the randomized alternative of Sec. 2.6.2 and
                           Sec. 5; Halko, Martinsson and Tropp 2011, Algorithm 4.2): Gaussian
                           sketch Y = A_pn Omega (Philox4x64-10 counter, keyed by sketch_seed, the
                           step and the cluster; 32 columns, doubled while the rank comes within
                           10 of them), column-pivoted QR of Y for the basis, rank = the first k
                           whose largest column of the remainder of A_pn falls below eps times its
                           largest column; coloured order only */
};

/* the sparsification transform (Sec. 2.6; the variants compared in the
 * ablation of Sec. 4.3) */
enum {
  SPAND_ORTHS = 0,  /* orthogonal transform after block scaling (Sec. 2.5,
                       2.6.1): Algorithm 2 */
  SPAND_INS = 1,    /* interpolative transform (Sec. 2.6.2) after block
                       scaling: the column-pivoted QR of A_np picks the kept
                       dofs c and T_cf = R_11^{-1} R_12 interpolates the
                       others, f, which are then eliminated; the f block
                       C_ff can fail to be positive definite (NOT_SPD) */
  SPAND_IN = 2      /* the same without the block scaling */
};

typedef struct spand_handle_s* spand_handle;

typedef struct {
  int32_t levels;     /* L of Algorithm 3: 2^(L-1) leaves; L >= 1 */
  double eps;         /* sparsification tolerance, >= 0 (0 = exact ND Cholesky) */
  int32_t skip;       /* no scaling / sparsification for the first `skip`
                         elimination steps counted from the leaves (Sec. 4.4) */
  int32_t precision;  /* SPAND_FP64, SPAND_FP32, SPAND_TF32 or SPAND_BF16 */
  int32_t maxit;      /* PCG iteration cap (paper: 500) */
  double tol;         /* PCG relative residual target (paper: 1e-12) */
  int32_t sparsify_order; /* SPAND_COLOURED or SPAND_SIMULTANEOUS */
  int32_t compression;    /* SPAND_CPQR or SPAND_RANDOMIZED */
  uint64_t sketch_seed;   /* seed of the Gaussian sketches (SPAND_RANDOMIZED) */
  int32_t variant;        /* SPAND_ORTHS, SPAND_INS or SPAND_IN; the
                             interpolative ones need the coloured order and
                             column-pivoted QR compression, and run their
                             sparsification in FP64 in every precision */
} spand_opts;

/* Fills *opts with levels 8, eps 1e-2, skip 0, FP64, maxit 500, tol 1e-10,
 * coloured sparsification order, column-pivoted QR compression, sketch seed 0,
 * the OrthS variant. */
void spand_default_opts(spand_opts* opts);

/*
 * spand_analyze -- host-only analysis (Algorithm 3, Sec. 2.3; clusters and
 * cluster trees, Sec. 2.3/2.7).
 *   n, rowptr, colind, vals : CSR of A (see conventions); vals is copied and
 *                             used by the next spand_factorize.
 *   coords                  : NULL, or n*dim float64 row-major vertex
 *                             coordinates (geometric separator); with NULL a
 *                             BFS level-set bisection is used.
 *   dim                     : coordinate dimension (ignored if coords NULL).
 *   opts                    : options (copied).
 *   out                     : receives a new handle (NULL on error).
 * Errors: SPAND_ERR_INVALID_ARG for a malformed CSR or options.
 */
int spand_analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                  const double* coords, int32_t dim, const spand_opts* opts, spand_handle* out);

/* One problem of a batch (the arguments of spand_analyze). */
typedef struct {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* vals;
  const double* coords;  /* NULL, or n*dim float64 row-major */
  int32_t dim;
} spand_problem;

/*
 * spand_analyze_batch -- spand_analyze of k independent problems (a batch of
 * systems that share nothing, e.g. many small diffusion problems solved
 * together), run on parallel host threads.
 *   k     : number of problems, >= 0.
 *   probs : k problem descriptions (host arrays, copied).
 *   opts  : k option sets, one per problem (levels usually differ with size).
 *   out   : k handles; on success every entry is a new handle, on any error
 *           every entry is NULL and no handle is left allocated.
 * Errors: those of spand_analyze; the message names the first failing
 * problem (lowest index).
 */
int spand_analyze_batch(int32_t k, const spand_problem* probs, const spand_opts* opts, spand_handle* out);

/*
 * spand_factorize -- numeric factorization on the current CUDA device
 * (Algorithm 2).  vals: NULL to use the values given to spand_analyze, or a
 * new float64[nnz] array for the same pattern (host or device memory).
 * Errors: SPAND_ERR_NOT_SPD (spand_get_stats gives the failing step/cluster),
 * SPAND_ERR_CUDA, SPAND_ERR_OOM.  A failed factorization leaves the handle
 * unfactorized.
 */
int spand_factorize(spand_handle h, const double* vals, void* cuda_stream);

/*
 * spand_solve -- PCG (Sec. 4) with z = M M^T r (Sec. 2.8).
 *   b       : float64[n] right-hand side (host or device), original ordering.
 *   x       : float64[n] solution (host or device), original ordering.
 *   iters   : optional, receives the number of products A p.
 *   relres  : optional, receives ||b - A x|| / ||b|| (true residual).
 * Errors: SPAND_ERR_STATE before a successful factorize;
 *         SPAND_ERR_NO_CONVERGENCE if maxit is reached above tol (x, iters and
 *         relres are still written).
 */
int spand_solve(spand_handle h, const double* b, double* x, int32_t* iters, double* relres,
                void* cuda_stream);

/*
 * spand_apply -- z = M M^T r, the preconditioner alone (Sec. 2.8), on device
 * vectors in the ORIGINAL ordering.  r and z are device float64[n]; they may
 * alias.
 */
int spand_apply(spand_handle h, const double* r_dev, double* z_dev, void* cuda_stream);

/*
 * spand_apply_noalloc -- the same z = M M^T r as spand_apply, for callers
 * that must not allocate device memory during the call: code running while
 * another component owns the device memory pool (for instance a framework's
 * caching allocator with a fixed budget), or a latency-critical loop where the
 * implicit device-wide synchronisation of cudaMalloc / cudaFree is not
 * acceptable.  The paper has no counterpart; this is a deployment variant.
 *   r_dev, z_dev : device float64[n], original ordering; they may alias.
 * Work space: one fixed array of 2^21 doubles (16 MiB) compiled into the
 * library, resident on every GPU that loads it until the process exits.  A
 * factorization whose apply needs more (n + its per-step temporaries + its
 * sparsification save area) is rejected with SPAND_ERR_INVALID_ARG before any
 * GPU work.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (nothing in
 * it needs to start at zero); calls whose GPU work overlaps -- on different
 * streams, handles or host threads -- race on it and must be serialised by the
 * caller.  Errors as spand_apply.
 */
int spand_apply_noalloc(spand_handle h, const double* r_dev, double* z_dev, void* cuda_stream);

/*
 * spand_sketch_gaussian -- the Gaussian test matrix of the randomized
 * compression of one interface (Sec. 2.6.2 names randomized methods for the
 * low-rank step): entry (i, j) of the m x ell matrix is a pure function of
 * (seed, step, cluster, i, j), drawn by Philox4x64-10 (Salmon et al., SC
 * 2011) under the key (seed, step * 2^32 + cluster) at the counter
 * (j, i / 4, 0, 0), with Box-Muller turning the block's four words into rows
 * 4 (i / 4) .. 4 (i / 4) + 3.  Column j is the same for every ell > j and
 * row i for every m > i.  No handle needed.
 *   out_dev     : device float64[m * ell], column-major (leading dimension m);
 *                 owned by the caller.
 *   cuda_stream : stream of the launch (asynchronous).
 * Errors: SPAND_ERR_INVALID_ARG for a negative step, cluster, m or ell, or a
 * null out_dev with m * ell > 0; SPAND_ERR_CUDA if the launch fails.
 */
int spand_sketch_gaussian(uint64_t seed, int32_t step, int32_t cluster, int32_t m, int32_t ell, double* out_dev,
                          void* cuda_stream);

/*
 * spand_sampled_outer -- out[e] = -lam[i] * x[j] for every stored entry e =
 * (i, j) of A, in the CSR order given to spand_analyze.  With x = A^{-1} b and
 * lam = A^{-1} (dL/dx) (the adjoint solve, same factorization since A is
 * SPD), this is dL/dA restricted to A's pattern (each stored value taken as
 * an independent parameter; for a symmetric parameterization add the entries
 * (i, j) and (j, i)).  Not part of the paper: it makes spand_solve
 * differentiable.
 *   lam_dev, x_dev : device float64[n]; out_dev : device float64[nnz].
 */
int spand_sampled_outer(spand_handle h, const double* lam_dev, const double* x_dev, double* out_dev,
                        void* cuda_stream);

/*
 * spand_get_tree -- the ordering and clusters (integer output of analyze).
 *   perm        : int32[n], perm[i] = vertex at position i (may be NULL)
 *   cluster_ptr : int32[n_clusters+1] (may be NULL)
 *   cluster_key : int32[3*n_clusters], (S, L, R) heap labels, none = -1
 *                 (may be NULL)
 *   n_clusters  : receives the number of clusters (required)
 *   n_steps     : receives L (may be NULL)
 * Call once with NULL arrays to size them.
 */
int spand_get_tree(spand_handle h, int32_t* perm, int32_t* cluster_ptr, int32_t* cluster_key,
                   int32_t* n_clusters, int32_t* n_steps);

/*
 * spand_get_step -- symbolic structure of elimination step t (1 = leaves ..
 * L = root).  Cluster indices are into that step's list.
 *   counts[5] (required): n_t, #children entries, #adj entries, #adjf entries,
 *                         #colours
 *   keys[3 n_t], child_ptr[n_t+1] / child_idx (indices into step t-1's list;
 *   step 1: the initial clusters), elim[n_t] (1 = eliminated at t),
 *   colour[n_t] (-1 if eliminated), adj_ptr[n_t+1] / adj_idx (cluster graph
 *   before the step), adjf_ptr[n_t+1] / adjf_idx (remaining clusters after the
 *   step's fill).  Any array may be NULL.
 */
int spand_get_step(spand_handle h, int32_t t, int32_t* counts, int32_t* keys, int32_t* child_ptr,
                   int32_t* child_idx, int32_t* elim, int32_t* colour, int32_t* adj_ptr,
                   int32_t* adj_idx, int32_t* adjf_ptr, int32_t* adjf_idx);

/*
 * spand_get_ranks -- after spand_factorize: cluster sizes of step t at its
 * start (sizes_before[n_t]) and after its sparsification (sizes_after[n_t];
 * equal to sizes_before where nothing was sparsified; 0 for eliminated
 * clusters).  Either array may be NULL.
 */
int spand_get_ranks(spand_handle h, int32_t t, int32_t* sizes_before, int32_t* sizes_after);

typedef struct {
  double t_analyze_s;     /* host analysis wall time */
  double t_factor_s;      /* last factorize wall time (stream-synchronous) */
  double t_solve_s;       /* last solve wall time */
  int32_t n_cg;           /* last solve iteration count */
  double relres;          /* last solve true relative residual */
  int64_t size_top;       /* size of the root separator right before elimination */
  int64_t mem_f;          /* stored factor entries (Sec. 4: mem_F) */
  double factor_flops;    /* algorithmic flops of the last factorization */
  double apply_bytes;     /* algorithmic bytes of one preconditioner apply */
  int32_t fail_step;      /* NOT_SPD: elimination step (1-based), else 0 */
  int32_t fail_cluster;   /* NOT_SPD: cluster index in that step, else -1 */
  int64_t device_bytes;   /* device memory held by the handle */
  int32_t apply_ctas_per_sm; /* shape of the preconditioner apply's cooperative
                                launch (CTAs per SM), chosen by the autotuner
                                at the first apply or set by
                                spand_set_apply_shape; 0 before the first apply */
} spand_stats;

int spand_get_stats(spand_handle h, spand_stats* st);

/* Per-phase device timings of the last factorization, summed over steps (ms):
 * out[0] eliminate, out[1] scale, out[2] sparsify, out[3] merge+assembly;
 * out[4] one preconditioner apply (last solve, mean), out[5] one SpMV + PCG
 * vector update (last solve, mean). */
int spand_get_phase_times(spand_handle h, double* out6);

/*
 * Kernel-family profile (for roofline reporting; not part of the method).
 * spand_set_profiling(h, 1) makes later factorize/solve/apply calls bracket
 * each batch of launches of one family with a CUDA event pair on the
 * launching stream (adds a few microseconds per batch).  Families:
 */
enum {
  SPAND_K_POTRF = 0,  /* pivot Cholesky tiles (Sec. 2.4, 2.5) */
  SPAND_K_TRSM = 1,   /* block-row triangular solves and pivot inverses */
  SPAND_K_SCHUR = 2,  /* Schur-complement update (Sec. 2.4) */
  SPAND_K_CPQR = 3,   /* sparsification QR (Sec. 2.6.1), all colours of a level */
  SPAND_K_COPY = 4,   /* merge gathers and transpose mirrors (Sec. 2.7) */
  SPAND_K_APPLY = 5,  /* one z = M M^T r (Sec. 2.8) */
  SPAND_K_PCG = 6     /* SpMV + fused PCG vector update, one iteration */
};
int spand_set_profiling(spand_handle h, int32_t on);
/* out4: batches' launches, summed device ms, algorithmic flops, algorithmic
 * bytes, accumulated since the last reset. */
int spand_get_kernel_profile(spand_handle h, int32_t family, double* out4);
int spand_reset_kernel_profile(spand_handle h);
/* Kernels launched by this handle since it was created (always counted). */
int spand_get_launch_count(spand_handle h, int64_t* launches);

/*
 * spand_set_apply_shape -- launch shape of the preconditioner apply (one
 * cooperative kernel for z = M M^T r): ctas_per_sm in 1..4 fixes the number
 * of CTAs per SM (capped by the kernel's occupancy); 0 (the default) lets the
 * library's autotuner choose at the first apply or solve after the handle's
 * first factorization, by timing every candidate on a scratch vector, and
 * keep that choice for the handle.  The shape never changes the result:
 * every item of an apply phase is computed by one CTA in a fixed order.
 */
int spand_set_apply_shape(spand_handle h, int32_t ctas_per_sm);

/*
 * spand_set_apply_wait -- failure-path knob (not part of the method).  The
 * preconditioner apply is one cooperative kernel whose phases are separated
 * by grid barriers; every barrier wait is bounded, and a wait that runs out
 * makes the CTA record the timeout and leave the kernel, so that the call
 * returns SPAND_ERR_TIMEOUT and the context stays usable.  For later
 * spand_apply / spand_apply_noalloc / spand_solve calls on h:
 *   polls       : polls per barrier wait before giving up (0 = the default,
 *                 2^24 polls with short sleeps, well over a second).
 *   unreachable : nonzero makes every barrier wait for one arrival more than
 *                 the grid has (a count nothing reaches), so every wait runs
 *                 out after `polls` polls and the call returns
 *                 SPAND_ERR_TIMEOUT without having computed z; 0 restores
 *                 normal barriers.
 */
int spand_set_apply_wait(spand_handle h, uint32_t polls, int32_t unreachable);

void spand_destroy(spand_handle h);

const char* spand_error_string(int code);
/* Message of the last failed call on this thread ("" if none). */
const char* spand_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPAND_H */
