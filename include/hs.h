/*
 * hs.h -- C ABI of libhs: CTMRG contraction of double-layer iPEPS tensor
 * networks in the Hermitian (bra-ket swap) basis, on one GB300 (sm_103a).
 *
 * Method: arXiv 2410.11596, "Exploiting the Hermitian symmetry in tensor
 * network algorithms". Each combined bra-ket leg of dimension D^2 is rotated
 * into the eigenbasis of the swap S (Sec. II.B); for real tensors the double
 * layer becomes Z2 block-sparse with an even sector of size D(D+1)/2 and an odd
 * sector of size D(D-1)/2, and the CTMRG contractions (Sec. II.A, Fig. 1(d))
 * become block GEMMs at about a quarter of the dense cost (Sec. II.B).
 *
 * Conventions used by every call
 * ------------------------------
 * - All pointers to tensor data are DEVICE pointers unless stated otherwise.
 *   The caller allocates and owns every input and output buffer; the context
 *   owns only its workspace, solver/BLAS handles and pinned staging memory.
 * - Every call enqueues its GPU work on the context's stream. Calls that must
 *   return host-visible results (sector sizes, status words) synchronise that
 *   stream before returning; this is stated per call.
 * - iPEPS tensor A: shape (d, D, D, D, D), legs (p, u, l, d, r), row-major,
 *   float64 (HS_F64) or interleaved complex128 (HS_C128).
 * - Combined bra-ket index of one double-layer leg: x = i + D * ibar with i
 *   the ket (from A) and ibar the bra (from conj A) index: the ket index runs
 *   fastest, as in the D = 2 listing of Sec. II.B.
 * - Hermitian basis of one leg (Sec. II.B): even states (k k') for k ascending,
 *   then (k l' + l k')/sqrt2 for k < l; odd states (k l' - l k')/sqrt2 for k < l.
 * - Sector-ordered block storage ("FSO"): a tensor with legs split into row
 *   legs and column legs is stored as the blocks of its block-diagonal matrix.
 *   A fused group of legs enumerates the parity tuples of its legs grouped by
 *   total parity (even group first), tuples in lexicographic order (first leg
 *   most significant), and inside a tuple the local indices row-major.
 *   Block p (p = 0 even, 1 odd) holds rows of fused parity p times columns of
 *   fused parity p, row-major; block 1 follows block 0. In the dense basis
 *   every leg is "all even" and the layout is the plain row-major matrix.
 * - Errors: no call aborts, exits or prints. Each returns an hs_status; the
 *   message of the last failure on the calling thread is hs_last_error().
 *   There is no CPU fallback: a missing capability is an error.
 */
#ifndef HS_H
#define HS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HS_ABI_VERSION 5

typedef enum {
  HS_OK = 0,
  HS_ERR_INVALID_ARG = -1,   /* null pointer, negative size, bad enum */
  HS_ERR_SHAPE = -2,         /* sizes inconsistent or above a limit */
  HS_ERR_DTYPE = -3,         /* dtype not supported by this call */
  HS_ERR_NOT_HERMITIAN = -4, /* odd blocks above tolerance where none may exist */
  HS_ERR_CUDA = -5,          /* a CUDA runtime call failed */
  HS_ERR_SOLVER = -6,        /* cuSOLVER / cuBLAS failure or non-zero info */
  HS_ERR_TIMEOUT = -7,       /* a bounded device wait gave up */
  HS_ERR_NONFINITE = -8,     /* NaN or Inf found in a result */
  HS_ERR_WORKSPACE = -9,     /* caller buffer smaller than required */
  HS_ERR_UNSUPPORTED = -10   /* valid request that this build does not implement */
} hs_status;

typedef enum { HS_F64 = 0, HS_C128 = 1 } hs_dtype;

/* Arithmetic of the block contractions (Sec. II.B). The normalisation, the
 * RDM traces and the projection of the new corner are FP64 in every mode;
 * the eigenvalues that choose the kept states are FP64 only with HS_EIG_F64
 * (HS_EIG_F32_PROJECTED and HS_EIG_SUBSPACE choose them from FP32
 * eigenvalues or FP32 Ritz values, see hs_eig_mode). */
typedef enum {
  HS_PREC_F64 = 0,    /* FP64 block GEMMs */
  HS_PREC_TF32X3 = 1, /* 3-pass split TF32 on tcgen05, FP32 accumulate */
  HS_PREC_TF32 = 2,   /* 1-pass TF32 on tcgen05, FP32 accumulate */
  HS_PREC_BF16X3 = 3  /* 3-pass split BF16 on tcgen05, FP32 accumulate */
} hs_precision;

/* Basis of the combined legs: dense (the plain combined basis, one sector)
 * or Hermitian (eigenbasis of S, two sectors). */
typedef enum { HS_BASIS_DENSE = 0, HS_BASIS_HERMITIAN = 1 } hs_basis;

/* How the projector of each parity block is computed (Sec. II.A: truncation
 * by an eigenvalue decomposition of the enlarged corner).
 * HS_EIG_F64: FP64 symmetric eigen-decomposition; C_new = diag(lambda_kept).
 * HS_EIG_F32_PROJECTED: FP32 eigen-decomposition chooses the kept states
 *   (by their FP32 eigenvalues) and their vectors; in FP64 the vectors are
 *   re-orthonormalised (two Loewdin steps, P <- (3/2 I - 1/2 P^T P)-updated)
 *   and the new corner is the FP64 projection C_new = P^T C' P (symmetric,
 *   not diagonal). Meant for the mixed-precision modes, whose C' carries FP32
 *   rounding already.
 * HS_EIG_SUBSPACE: as HS_EIG_F32_PROJECTED, but the kept vectors come from a
 *   warm-started block subspace iteration on each parity block (products H X
 *   in the environment's precision, on tcgen05 or the FP64 kernel; the warm
 *   rows re-orthonormalised by a Loewdin step;
 *   unconverged rounds take a Chebyshev-filtered step, orthonormalised by
 *   Cholesky-QR and a Loewdin step; Rayleigh-Ritz of size m = k + max(24, k/3),
 *   at most 192, by an FP32 Jacobi eigensolver; at most 8 rounds, fewer when
 *   the residual stalls far from the tolerance) seeded with the previous
 *   move's subspace (kept plus oversampled vectors). Converged when every
 *   Ritz pair that can be kept has residual |H x - theta x| <= tol max|theta|
 *   (tol = 1e-6 with FP64 products, 1e-5 with tensor-core products), or, with
 *   tensor-core products, when a round has stalled below 10 tol (less than a
 *   factor 2 better than the previous round: the rounding floor of the
 *   products, 1e-5..3e-5 at D = 7);
 *   such a floor then serves as the tolerance of the following moves (times
 *   1.5) until a round gets below tol again. Otherwise, on the first move, or
 *   when the sector sizes cannot be carried over, the move falls back to
 *   HS_EIG_F32_PROJECTED. With tensor-core products, where the Cholesky-QR
 *   of a filtered basis breaks down, the round is run again on a
 *   Householder-QR basis instead. Kept vectors carry a canonical sign
 *   (largest entry positive) so that the gauge, and with it the warm start,
 *   is stationary at the fixed point; while the environment still moves (the
 *   move's first residual above 1e-3) they are instead ordered and signed
 *   like the previous move's kept vectors they overlap most (overlap above
 *   1/2, per parity block).
 * HS_EIG_SUBSPACE_ADAPTIVE: as HS_EIG_SUBSPACE, with the residual tolerance of
 *   each move set by how much the environment still changes: tol = 0.1 delta
 *   clamped to [1e-5 (1e-6 with FP64 products), 1e-3], delta the residual of the
 *   warm start in the previous move's first round (how far the kept subspace
 *   turned in one move). While the environment moves (the first moves after
 *   the start) the projector is found only to that accuracy; at the fixed
 *   point delta falls to the rounding level and the tolerance is
 *   HS_EIG_SUBSPACE's. Intermediate environments then differ from an
 *   exact-eigensolver run by about delta; the fixed point does not. */
typedef enum { HS_EIG_F64 = 0, HS_EIG_F32_PROJECTED = 1, HS_EIG_SUBSPACE = 2, HS_EIG_SUBSPACE_ADAPTIVE = 3 } hs_eig_mode;

/* Which library runs the FP64 block GEMMs (HS_PREC_F64 only). */
typedef enum { HS_GEMM_OWN = 0, HS_GEMM_CUBLAS = 1 } hs_gemm_backend;

typedef struct hs_ctx_s* hs_ctx;

/* The double-layer tensor a[u, l, d, r] (Sec. II.A, Fig. 1(b)) in FSO storage
 * with row legs (u, l) and column legs (d, r), all four legs of dimension D^2
 * split (n_even, n_odd). Only the even-total blocks exist for real A. There is
 * no block-offset table: the FSO order fixes every block's position (block 1
 * starts after the rows(0) x cols(0) entries of block 0, and inside a block the
 * parity tuples follow in lexicographic order), so the sector sizes are the
 * whole descriptor.
 *
 * Complex A (dtype HS_C128) in the Hermitian basis (Sec. II.C): every block of
 * a in the eigenbasis of S is purely real (even total parity) or purely
 * imaginary (odd). Such "graded" tensors, and the environment built from
 * them, are stored as ONE dense row-major real matrix over the same row and
 * column leg groups, rows and columns each in FSO order (even group first);
 * an entry of odd total parity holds the imaginary part, an even one the real
 * part. Products follow the sign rule of Eq. (2)-(3).
 * Complex A in the dense basis (the comparison path, nothing of the symmetry
 * used): the plain double layer, interleaved complex128, (D^2)^4 entries. */
typedef struct {
  int D;                 /* bond dimension of A */
  int n_even, n_odd;     /* per-leg sector sizes: (D(D+1)/2, D(D-1)/2) or (D^2, 0) */
  hs_basis basis;
  hs_dtype dtype;        /* HS_F64 (Z2 blocks) or HS_C128 (graded dense matrix, below) */
  double* data;          /* device, caller-owned */
  size_t capacity_bytes; /* size of data */
  /* HOTRG tensors: sectors of the vertical legs (u, d) and of the horizontal
   * legs (l, r). The double-layer calls set both to (n_even, n_odd). */
  int v_even, v_odd, h_even, h_odd;
} hs_z2_tensor;

/* The C4v environment (Sec. II.A, Fig. 1(d)): one corner C[chi, chi] and one
 * edge T[alpha, x, beta]. Both are FP64 in FSO storage:
 *   C: row leg beta, column leg gamma (block diagonal);
 *   T: row legs (alpha, x), column leg beta.
 * Complex environments (dtype HS_C128) are graded (see hs_z2_tensor) and
 * oriented: boundary tensors run clockwise, alpha/beta of T and the row/column
 * of C are the incoming/outgoing legs, and C is not symmetric.
 * The boundary leg has sectors (chi_even, chi_odd). Buffers are caller-owned,
 * sized with hs_env_bytes(). Fields other than C, T and the byte counts are
 * written by the library. */
typedef struct {
  int D, chi_max;
  int chi_even, chi_odd; /* current boundary sectors (host copy) */
  int q_even, q_odd;     /* sectors of the double-layer legs */
  hs_basis basis;
  hs_precision precision;
  hs_gemm_backend gemm_backend;
  int moves;             /* moves done since hs_ctmrg_init */
  double log_norm_C, log_norm_T; /* logs of the last normalisation factors */
  double* C;             /* device, caller-owned */
  double* T;             /* device, caller-owned */
  size_t C_bytes, T_bytes;
  hs_eig_mode eig_mode;  /* set to HS_EIG_F64 by hs_ctmrg_init; the caller may change it between moves */
  hs_dtype dtype;        /* HS_F64, or HS_C128 for a complex double layer (graded storage, below) */
} hs_env;

/* Per-move record filled by hs_ctmrg_move (host memory). */
typedef struct {
  int chi_even, chi_odd; /* sectors kept */
  int n_even, n_odd;     /* sizes of the two eigenproblems (dense basis: n_odd = 0) */
  double lam_max;        /* largest |eigenvalue| of the enlarged corner */
  double lam_cut;        /* smallest |eigenvalue| kept */
  double lam_next;       /* largest |eigenvalue| discarded (0 if none) */
  double gap;            /* (lam_cut - lam_next) / lam_max, +inf if nothing discarded */
  double log_norm_C, log_norm_T;
  double gemm_flops;     /* sum over block GEMMs of 2 M N K in this move */
  int flags;             /* bit 0: gap below 1e-9 (degenerate cut); bit 1: the subspace
                            eigensolver converged (no fallback); bit 2: it fell back */
  int subspace_iters;    /* Rayleigh-Ritz rounds of the subspace eigensolver (0 if unused) */
  int subspace_reason;   /* 0 converged, 1 no warm start, 2 sector sizes changed, 3 subspace too
                            large, 4 Cholesky failure (non-positive pivot), 5 not converged, 6 selection
                            at the edge of the subspace, 7 Rayleigh-Ritz eigensolver failure; -1 not
                            used */
  double subspace_resid; /* largest residual / max|theta| over the candidates in the last round */
} hs_move_info;

typedef enum { HS_RDM_TWO_SITE = 0, HS_RDM_ENV_ONE_SITE = 1, HS_RDM_ONE_SITE = 2 } hs_rdm_kind;

/* Per-step record of hs_hotrg_step (host memory). */
typedef struct {
  int h_even, h_odd;     /* sectors kept on the truncated legs */
  int side;              /* 0: left Gram matrix supplied the isometry, 1: right; a horizontal
                            step works on the tensor turned by 90 degrees, R[u,l,d,r] =
                            T[l,d,r,u], so there 0 is T's upper legs and 1 its lower ones */
  double discarded_left, discarded_right; /* discarded eigenvalue weight of each Gram matrix */
  double log_norm;       /* log of the max-abs normalisation of the new tensor */
  double trace;          /* sum_{u,l} T[u,l,u,l] of the new (normalised) tensor */
} hs_hotrg_info;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device` using `stream` (a cudaStream_t;
 * NULL selects the legacy default stream). */
hs_status hs_create(hs_ctx* out, int device, void* stream);
hs_status hs_destroy(hs_ctx ctx);
/* Message of the last failure on this thread ("" if none). Never NULL. */
const char* hs_last_error(void);
/* Block until all work of the context has finished; reports deferred
 * device-side errors. */
hs_status hs_sync(hs_ctx ctx);
int hs_abi_version(void);

/* ---- double layer and Hermitian basis (Sec. II.A, II.B) --------------- */

/* a[x_u, x_l, x_d, x_r] = sum_p A[p,u,l,d,r] conj(A[p,ubar,lbar,dbar,rbar])
 * (Fig. 1(b)) in the plain combined basis, dense row-major (D^2)^4 into a_out
 * (device, caller-owned, (D^2)^4 doubles; complex: interleaved complex128).
 * A is device memory. Asynchronous. */
hs_status hs_make_double_layer(hs_ctx ctx, const double* A, int d, int D, hs_dtype dtype,
                               double* a_out);

/* Bytes of an hs_z2_tensor for bond dimension D in the given basis; 0 when D < 1 or dtype is
 * neither HS_F64 nor HS_C128. */
size_t hs_z2_tensor_bytes(int D, hs_basis basis, hs_dtype dtype);

/* Rotate a dense double layer (layout of hs_make_double_layer, device) into
 * the eigenbasis of S on all four legs, a~ = (U^T)^{x4} a (Sec. II.B), and
 * store the even-total blocks in out (FSO, fields D/n_even/n_odd/basis set
 * here; out->data and out->capacity_bytes set by the caller). The odd-total
 * blocks are computed too: if their largest modulus exceeds
 * herm_tol * max|a~| the call returns HS_ERR_NOT_HERMITIAN. Synchronises. */
hs_status hs_to_hermitian_basis(hs_ctx ctx, const double* a_dense, int D, hs_dtype dtype,
                                double herm_tol, hs_z2_tensor* out);

/* Inverse of hs_to_hermitian_basis (Sec. II.B): a = U^{x4} a~ from the stored
 * blocks of a double layer in the Hermitian basis (t: HS_F64 Z2 blocks, or a
 * HS_C128 graded tensor) into a_dense (device, caller-owned, (D^2)^4 doubles
 * in the layout of hs_make_double_layer; interleaved complex128 for
 * HS_C128). HS_ERR_SHAPE if t's sectors are not those of a double layer of
 * bond dimension t->D (a HOTRG tensor after truncation). Asynchronous. */
hs_status hs_from_hermitian_basis(hs_ctx ctx, const hs_z2_tensor* t, double* a_dense);

/* Fused form of the two calls above: from A (device; real, or interleaved
 * complex128 with dtype HS_C128) straight to the stored blocks of a~ in
 * `basis` (HS_BASIS_DENSE gives the plain layout).
 * dtype HS_C128 writes the graded a~ in the Hermitian basis (Sec. II.C), and
 * the plain complex double layer (interleaved complex128) in the dense basis.
 * Asynchronous. */
hs_status hs_double_layer_hermitian(hs_ctx ctx, const double* A, int d, int D, hs_dtype dtype,
                                    hs_basis basis, hs_z2_tensor* out);

/* ---- CTMRG (Sec. II.A, Fig. 1(d)) ------------------------------------- */

/* Bytes needed for env->C and env->T at bond dimension D and chi_max (real
 * environments and graded complex ones; complex environments of the dense
 * basis, interleaved complex128, need twice these). */
hs_status hs_env_bytes(int D, int chi_max, size_t* C_bytes, size_t* T_bytes);

/* Traced-boundary initial environment: the open outer legs of the first
 * corner and edge are closed with delta(i, ibar) = sum_k |k k'>, an even
 * state, so C0 = a(delta, delta, ., .) and T0 = a(., delta, ., .) with chi0 =
 * D^2. Sets every library-written field of env. Asynchronous. */
hs_status hs_ctmrg_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_precision precision,
                        hs_gemm_backend backend, hs_env* env);

/* One C4v CTMRG move: enlarged corner C' = T C T a (block GEMMs), one FP64
 * symmetric eigen-decomposition per parity block, the chi eigenvalues of
 * largest modulus kept across both blocks (ties: larger |lambda|, then the
 * even block, then the lower eigenvalue), C <- diag(lambda_kept),
 * T <- P^T (T a) P, then C and T divided by their largest modulus.
 * Complex environments (HS_C128): graded block GEMMs (FP64), then the chi
 * largest singular values of C' = U S V^dagger, found as the top
 * eigenvectors of H = M M^T with C' = J M J (J = diag(1, i) by parity; one
 * eigen-decomposition of size chi*D^2, FP64 for HS_EIG_F64, FP32 followed by
 * two FP64 Loewdin steps for HS_EIG_F32_PROJECTED; the subspace modes run the
 * warm-started subspace iteration on H as one block, with the tolerances of
 * the real path, falling back to the FP32 decomposition); C <- U^dagger C' U,
 * T <- U^dagger (T a) U; the new boundary sectors are (chi, 0). lam_* in info
 * are singular values. The graded GEMMs and H run in the environment's
 * precision (FP64 kernel or tcgen05).
 * Complex environments of the dense basis (the comparison path): the same
 * truncation with plain complex tensors, each complex product four FP64 GEMMs,
 * U from the complex Hermitian FP64 eigen-decomposition of C' C'^dagger; only
 * HS_PREC_F64 with HS_EIG_F64 (else HS_ERR_UNSUPPORTED).
 * info (host, may be NULL) receives the move record. Synchronises once
 * (to learn the new sector sizes). */
hs_status hs_ctmrg_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env* env, int chi,
                        hs_move_info* info);

/* One move of each of n independent CTMRG instances (any mix of D, chi and
 * dtype), concurrently: instance i runs hs_ctmrg_move(ctxs[i], a[i],
 * env[i], chi[i], &info[i]) on its own context, whose stream and workspace
 * no other instance may share, from a pool of nthreads host threads (1 to
 * 256), so that the GPU overlaps the instances' kernels. info (host, n
 * records) and ms (host, n wall-clock latencies in milliseconds) may be NULL.
 * Returns when all instances are done; on failures, every instance still
 * runs and the first failing instance's status and message are returned.
 * The paper has no counterpart: this is the batched execution of many
 * independent networks. */
hs_status hs_ctmrg_move_batched(hs_ctx* ctxs, int n, const hs_z2_tensor* const* a, hs_env* const* env,
                                const int* chi, hs_move_info* info, double* ms, int nthreads);

/* Copy the environment out in the plain dense layout: C_dense[chi, chi] and
 * T_dense[chi, D^2, chi] (device, caller-owned, FP64; interleaved complex128
 * for HS_C128 environments), with the boundary leg ordered as stored (even
 * sector first) and the double-layer leg rotated back to the plain combined
 * basis. Asynchronous. */
hs_status hs_env_to_dense(hs_ctx ctx, const hs_env* env, double* C_dense, double* T_dense);

/* ---- Directional CTMRG: four corners, four edges, no lattice symmetry -----
 *
 * Sec. II.A runs CTMRG with C4v symmetry "for simplicity". Without it the
 * environment of a one-site unit cell has four corners and four edges, and a
 * directional move grows one side by a column of double-layer tensors and
 * truncates its bonds back with oblique projectors from the SVD of the two
 * quarters (enlarged corners) on that side: X = Q1^T Q4^T = U S V^T, keep the
 * chi largest singular values (and only those above 1e-12 s_max),
 * P_a = Q4^T V S^-1/2 above each truncated bond, P_b = Q1 U S^-1/2 below it.
 * In the Hermitian basis every tensor is Z2 block-sparse (Sec. II.B) and the
 * SVD splits into one per parity block; the kept states are the chi largest
 * over both blocks. FP64 GEMMs and FP64 SVD (hs_svd_mode). Real double
 * layers only (HS_F64).
 *
 * Bonds: 0 top, 1 right, 2 bottom, 3 left side of the boundary. Corner k
 * (C1 upper left, C2 upper right, C3 lower right, C4 lower left) joins bond
 * k-1 (mod 4, its incoming leg) to bond k (outgoing); edge k (T1 top, T2 right,
 * T3 bottom, T4 left) has both ends on bond k and its bulk leg on the
 * double-layer leg facing it (up, right, down, left). Legs run clockwise
 * around the lattice: T1[alpha, x, beta] left to right, T2 top to bottom, T3
 * right to left, T4 bottom to top. Storage: C[k] is the Z2 matrix
 * [in | out], T[k] the Z2 matrix [(alpha, x) | beta], both in FSO block
 * order (hs_z2_tensor). */
/* SVD of the directional move's parity blocks: one-sided Jacobi (cuSOLVER
 * gesvdj; singular values to about 1e-14 of the largest) or the polar-
 * decomposition SVD (cuSOLVER Xgesvdp; 4-8 times faster on these blocks,
 * singular values to about 1e-11..1e-9 of the largest). */
typedef enum { HS_SVD_JACOBI = 0, HS_SVD_POLAR = 1 } hs_svd_mode;

typedef struct {
  int D, chi_max;
  int chi_even[4], chi_odd[4]; /* sectors of the four boundary bonds (host copy) */
  int q_even, q_odd;           /* sectors of the double-layer legs */
  hs_basis basis;
  int moves;                   /* directional moves since hs_ctmrg4_init (a sweep is four) */
  double* C[4];                /* device, caller-owned; C_bytes each */
  double* T[4];                /* device, caller-owned; T_bytes each */
  size_t C_bytes, T_bytes;     /* at least hs_env_bytes(D, chi_max) */
  double log_norm_C[4], log_norm_T[4]; /* logs of the last normalisation factors */
  hs_svd_mode svd;             /* set to HS_SVD_JACOBI by hs_ctmrg4_init; may change between moves */
} hs_env4;

typedef struct {
  int direction;          /* side moved: 0 left, 1 top, 2 right, 3 bottom */
  int chi_even, chi_odd;  /* sectors kept on the moved side's bond */
  int m_even, m_odd;      /* rows of the two SVD blocks (the side's first neighbour bond x bulk leg) */
  int n_even, n_odd;      /* columns (the side's other neighbour bond x bulk leg) */
  double s_max, s_cut, s_next; /* largest, smallest kept and largest discarded singular value */
  double gap;             /* (s_cut - s_next) / s_max, +inf if nothing discarded */
  double gemm_flops;      /* sum over block GEMMs of 2 M N K in this move */
} hs_move4_info;

/* Traced-boundary initialisation of all eight tensors from the double layer a
 * (HS_F64, either basis; every bond starts at the double-layer leg's sectors),
 * each divided by its largest modulus. Caches the four rotated copies of a in
 * the context; a must not change until the next hs_ctmrg4_init. One context
 * serves the directional runs of one double layer at a time: after another
 * hs_ctmrg4_init with a different a, a move given the earlier a fails with
 * HS_ERR_INVALID_ARG. */
hs_status hs_ctmrg4_init(hs_ctx ctx, const hs_z2_tensor* a, int chi_max, hs_env4* env);

/* One directional move of side `direction` (0 left, 1 top, 2 right, 3 bottom;
 * a sweep is 0, 1, 2, 3): updates the side's two corners and its edge, with
 * chi (<= env->chi_max) states kept on its bond. sv_out (host, may be NULL,
 * at least chi entries) receives the kept singular values divided by the
 * largest, descending. Synchronises the stream once (the kept sector sizes
 * fix the shapes that follow). HS_ERR_SOLVER if the SVD does not converge,
 * HS_ERR_NONFINITE if a normalisation factor is not finite. */
hs_status hs_ctmrg4_move(hs_ctx ctx, const hs_z2_tensor* a, hs_env4* env, int chi, int direction,
                         hs_move4_info* info, double* sv_out);

/* Dense copies of the eight tensors (device, caller-owned, FP64): C_dense[k]
 * [in bond, out bond] and T_dense[k] [bond, D^2, bond], boundary legs ordered
 * as stored (even sector first), the bulk leg rotated back to the plain
 * combined basis. Asynchronous. */
hs_status hs_env4_to_dense(hs_ctx ctx, const hs_env4* env, double* const* C_dense, double* const* T_dense);

/* ---- HOTRG (Sec. II.A, Ref. xie12) ------------------------------------ */

/* Bytes of a HOTRG tensor buffer for bond dimension D and chi: max(D^2, chi)^4 doubles; 0 when
 * D < 1 or chi < 1. */
size_t hs_hotrg_tensor_bytes(int D, int chi);

/* Start a HOTRG run: copy the double layer a (FSO) into t (caller-owned,
 * t->data with hs_hotrg_tensor_bytes) and divide it by its largest modulus;
 * *log_norm (host) receives the log of that factor. Synchronises. */
hs_status hs_hotrg_init(hs_ctx ctx, const hs_z2_tensor* a, hs_z2_tensor* t, double* log_norm);

/* One HOTRG coarse-graining step on t (in place). direction 0 stacks two
 * tensors vertically and truncates the fused horizontal legs to chi;
 * direction 1 does the same on the tensor turned by 90 degrees (horizontal
 * stacking). The isometry is the top-chi eigenvector set of the left or the
 * right Gram matrix of the fused leg, whichever discards less weight (ties:
 * left); one FP64 eigen-decomposition per parity block, states kept across
 * both blocks by eigenvalue. The new tensor is divided by its largest
 * modulus. precision: HS_PREC_F64 runs the block GEMMs on the FP64 kernel;
 * HS_PREC_TF32X3 / TF32 / BF16X3 run them on tcgen05 (operands split straight
 * from their source layouts, FP32 accumulation, FP64 output); the Gram
 * eigen-decompositions are FP64 in every precision. info (host, may be NULL)
 * receives the step record. Synchronises. */
hs_status hs_hotrg_step(hs_ctx ctx, hs_z2_tensor* t, int chi, int direction, hs_precision precision,
                        hs_hotrg_info* info);

/* Free energy per site of a HOTRG run (Sec. II.A, Ref. xie12), host only:
 *   ln Z / N = ln c_0 + sum_{k=1..steps} ln(c_k) / 2^k + ln Tr(T_steps) / 2^steps,
 * with log_norms[0] = ln c_0 from hs_hotrg_init, log_norms[k] = ln c_k the
 * log_norm of step k (host array of steps + 1 values) and trace the `trace`
 * of the last step's hs_hotrg_info. *log_z (host) receives the value.
 * HS_ERR_INVALID_ARG on null pointers or steps < 1; HS_ERR_NONFINITE if
 * trace is not positive and finite, or the result is not finite. */
hs_status hs_hotrg_log_z(const double* log_norms, int steps, double trace, double* log_z);

/* ---- observables (Sec. III.A) ----------------------------------------- */

/* HS_RDM_TWO_SITE: rho[(s1 s2), (s1' s2')] of a horizontal bond from the
 * environment and A (device; real, or interleaved complex128 with HS_C128),
 * not normalised, into out (device, d^4 doubles); then tr_out[0] = Tr rho and
 * tr_out[1] = Tr(rho h) with h a d^2 x d^2 real matrix (device). In the Hermitian basis only the S-even part of the
 * open double layer meets the Z2-even environment, so rho is Hermitian by
 * construction; the entries are computed for (row <= col) and mirrored.
 * HS_RDM_ENV_ONE_SITE: the one-site environment eps[u, l, d, r] (Eq. (4)),
 * (D^2)^4 doubles in the plain combined basis; h and tr_out unused.
 * HS_RDM_ONE_SITE: the one-site reduced density matrix rho1[s, s'] =
 * sum eps[x_u, x_l, x_d, x_r] A[s, ket(x)] conj(A[s', bra(x)]) (d^2 doubles,
 * not normalised); tr_out[0] = Tr rho1, tr_out[1] = Tr(rho1 h) with h a d x d
 * real matrix (device, may be NULL).
 * HS_C128 (complex A, interleaved; graded environment): rho, eps and the
 * traces are interleaved complex128 (tr_out: Re/Im of Tr rho, then of
 * Tr(rho h)), computed in complex arithmetic on the clockwise boundary ring.
 * Asynchronous. */
hs_status hs_rdm(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_dtype dtype,
                 hs_rdm_kind kind, const double* h, double* out, double* tr_out);

/* Normalised corner spectrum (Sec. III.A): the singular values of the corner
 * C of env divided by the largest, in descending order, into out (device,
 * chi_even + chi_odd doubles). Real environments: one FP64 SVD per parity
 * block of the block-diagonal C, merged. Complex (graded) environments: C =
 * J M J with J = diag(1, i) by parity, so the values are those of the real M
 * (the stored matrix with its odd-odd block negated). Synchronises (to check
 * the solver's status). */
hs_status hs_corner_spectrum(hs_ctx ctx, const hs_env* env, double* out);

/* Correlation length of a real C4v environment: xi = -1/ln|lambda_2/lambda_1|
 * of the column transfer matrix E[(alpha,l,beta),(alpha',r,beta')] =
 * sum_{u,d} T[alpha,u,alpha'] a[u,l,d,r] T[beta',d,beta] (top edge left to
 * right, bottom edge right to left), from A (device, real, the tensor the
 * environment was built from). E is symmetric for real C4v tensors; a Lanczos
 * iteration with full re-orthogonalisation (at most max_iter matvecs, 4 to
 * 400; each is three GEMMs in the plain combined basis, in the environment's
 * precision) runs until the two largest |Ritz values| change by at most
 * tol * lambda_1. lam_out (host, 2) receives |lambda_1| and |lambda_2|;
 * xi_out (host) xi (0 if lambda_2 = 0, +inf if degenerate). Complex
 * environments: HS_ERR_UNSUPPORTED. Not converged: HS_ERR_TIMEOUT with the
 * last estimates written. Synchronises. */
hs_status hs_correlation_length(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, int max_iter,
                                double tol, double* lam_out, double* xi_out);

/* ---- profiling ------------------------------------------------------- */

/* Phases of hs_ctmrg_move timed with CUDA events on the context stream. */
typedef enum {
  HS_PHASE_GEMM = 0,      /* block GEMMs (own kernels or cuBLAS) */
  HS_PHASE_PERMUTE = 1,   /* leg permutations between block layouts */
  HS_PHASE_EIG = 2,       /* per-block symmetric eigen-decompositions */
  HS_PHASE_SELECT = 3,    /* choice of kept states, projector gather, new corner */
  HS_PHASE_NORMALIZE = 4, /* max-abs normalisation of the edge */
  HS_PHASE_GEMM_TC = 5,   /* block GEMMs on the tensor cores (TF32/BF16 modes) */
  HS_PHASE_GEMM_TC_SPLIT = 6, /* those of them whose epilogue writes the next GEMM's permuted split
                                 operand (the enlarged corner and edge products); also in phase 5 */
  HS_PHASE_COUNT = 7
} hs_phase;

/* Turn per-phase timing on (1) or off (0); either way the counters reset.
 * Timing adds events between phases but changes no computation. */
hs_status hs_profile_enable(hs_ctx ctx, int enable);

/* Restrict the per-phase timing to the phases whose bit is set in mask
 * (bit i = phase i; all phases by default). Each timed phase adds two events
 * to the stream, so timing fewer phases perturbs a launch-bound move less.
 * Errors: HS_ERR_INVALID_ARG for a bad context. */
hs_status hs_profile_phases(hs_ctx ctx, unsigned mask);

/* Read the counters accumulated since the last reset: phase_ms[i] and
 * phase_flops[i] (host, n_phases entries: milliseconds of device time and
 * algorithmic flops, sum of 2 M N K over the block GEMMs, per phase) and
 * launches (number of this library's own kernel launches; library calls such
 * as cuSOLVER and cuBLAS are not counted). Any output pointer may be NULL. */
hs_status hs_profile_read(hs_ctx ctx, double* phase_ms, double* phase_flops, int n_phases,
                          long long* launches);

/* ---- block GEMM primitive (Sec. II.B) --------------------------------- */

/* C[M, N] = A[M, K] B[N, K]^T for row-major FP64 device matrices with leading
 * dimensions lda >= K, ldb >= K, ldc >= N: the dense GEMM that the Z2 block
 * contraction performs inside one parity block. HS_PREC_F64 runs the FP64
 * kernel; the TF32/BF16 modes split A and B into hi/lo parts (padded copies in
 * the context workspace) and run the tcgen05 tensor-core kernel with FP32
 * accumulation, writing FP64. Asynchronous; a timed-out device wait is
 * reported by the next hs_sync as HS_ERR_TIMEOUT. */
hs_status hs_gemm(hs_ctx ctx, hs_precision precision, int M, int N, int K, const double* A, int lda,
                  const double* B, int ldb, double* C, int ldc);

/* ---- block GEMM without allocation ------------------------------------ */

/* The tensor-core block GEMM of hs_gemm (TF32X3, TF32 or BF16X3; C = A B^T,
 * FP64 row-major device matrices) for callers that must not allocate device
 * memory: applications whose own memory manager owns all device memory,
 * latency-critical loops that cannot take the synchronisation cudaMalloc and
 * cudaFree may imply, and plugins that may not change the device memory
 * footprint. The paper has no counterpart; this is a service of the library.
 * It takes no context and allocates nothing: its scratch (the split, padded
 * operands) is a static device array of 16 MiB that every GPU which loads the
 * library holds until exit, so 2 (M + N) Kp e <= 16 MiB is required (Kp = K
 * rounded up to 32 for TF32 modes or 64 for BF16X3; e = 4 or 2 bytes);
 * larger requests return HS_ERR_SHAPE. The first call on each device looks the
 * array's device address up (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the array:
 * calls whose GPU work overlaps race, so order them on one stream.
 * status_out (device int, required) is set to 0 and receives a non-zero code
 * if a bounded wait in the kernel gave up. stream is a cudaStream_t (NULL:
 * legacy default stream). Asynchronous. */
hs_status hs_gemm_static(hs_precision precision, int M, int N, int K, const double* A, int lda,
                         const double* B, int ldb, double* C, int ldc, int* status_out, void* stream);

/* Adjoint of the two-site RDM with the environment held fixed (the
 * differentiation pattern of the hot path; the paper has no formula for it):
 * dA[p,u,l,d,r] = sum_{IJ} drho[I,J] d rho[I,J] / d A[p,u,l,d,r] for the rho
 * of hs_rdm(HS_RDM_TWO_SITE) before any mirroring (its exact mathematical
 * derivative). drho: device, d^4 doubles, layout of rho; dA_out: device,
 * d*D^4 doubles. Complex A (HS_C128, graded environment): A, drho and dA_out
 * interleaved complex128, drho the cotangent dE/dRe rho + i dE/dIm rho and
 * dA_out = dE/dRe A + i dE/dIm A. Asynchronous. */
hs_status hs_rdm_vjp(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_dtype dtype,
                     const double* drho, double* dA_out);

/* Gradient of the bond energy E = Re Tr(rho h) / Tr rho (rho of
 * hs_rdm(HS_RDM_TWO_SITE), environment held fixed): dA_out = dE * dE/dA for
 * real A, dE * (dE/dRe A + i dE/dIm A) for complex A (interleaved). The
 * cotangent of rho, dE (conj(1/Tr rho) h^T - conj(Tr(rho h)/(Tr rho)^2) I), is
 * formed on the device from the traces of the same forward contraction, then
 * the reverse pass of hs_rdm_vjp runs. h: device, d^2 x d^2 real (required).
 * The paper has no formula for it (differentiation of the hot path).
 * Asynchronous. */
hs_status hs_energy_vjp(hs_ctx ctx, const hs_env* env, const double* A, int d, int D, hs_dtype dtype,
                        const double* h, double dE, double* dA_out);

/* Energy of a whole C4v CTMRG run and its gradient through the iterations:
 * from A (device, real, (d, D, D, D, D)) the double layer in `basis`, the
 * traced-boundary environment, `moves` moves of hs_ctmrg_move with FP64 block
 * GEMMs and the FP64 eigen-decomposition (chi kept states), then the bond
 * energy E = Tr(rho h) / Tr rho of the two-site RDM (h: device, d^2 x d^2 real);
 * *energy_out (host) receives E and dA_out (device, d D^4 doubles) dE/dA,
 * by a reverse pass over every step (the adjoint of the symmetric
 * eigen-decomposition for the projectors, of the block GEMMs and permutations,
 * of the initialisation and the double layer). The derivative is the one
 * along C4v-symmetric changes of A (the C4v CTMRG reads one triangle of the
 * enlarged corner), and it needs distinct eigenvalues around the cut. The
 * paper has no formula for it (the variational use of CTMRG environments it
 * refers to in Sec. III.A). Allocates its tape, synchronises. */
hs_status hs_ctmrg_energy_grad(hs_ctx ctx, const double* A, int d, int D, hs_basis basis, int chi, int moves,
                               const double* h, double* energy_out, double* dA_out);

/* A planning estimate of a context's largest work buffers for (D, chi): the
 * two ping-pong buffers of the enlarged-corner and edge chains, sized for the
 * plain basis ((chi D^2)^2 doubles each, chi at least D^2), and three
 * chi^2 D^2 buffers. Not counted: solver workspaces, tensor-core split
 * operands and the subspace solver's buffers. precision is not used yet.
 * HS_ERR_INVALID_ARG if D or chi is below 1 or bytes is NULL. Host only. */
hs_status hs_workspace_query(int D, int chi, hs_precision precision, size_t* bytes);

/* Diagnostic: runs the tensor-core GEMM's bounded mbarrier wait (the wait
 * every pipeline stage of that kernel uses, which gives up after a fixed
 * number of try_wait rounds, raises the kernel's abort flag and records an
 * error code) on barriers whose outcome is known, with `limit` rounds
 * (1 <= limit <= the kernel's own limit). result (host, 7 ints): wait on a
 * barrier nothing completes -> {0 (gave up), 7 (code recorded), 1 (abort
 * raised)}; wait with the abort flag raised -> {0, 0 (nothing recorded)};
 * wait on a barrier completed by one arrival -> {1, 0}. Synchronises. */
hs_status hs_selftest_bounded_wait(hs_ctx ctx, long long limit, int* result);

#ifdef __cplusplus
}
#endif
#endif /* HS_H */
