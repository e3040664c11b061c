/*
 * ipeps_ctm.h -- C ABI of the GB300 CTM library.
 *
 * The library contracts the infinite double-layer network of an iPEPS with
 * the corner transfer matrix (CTM) renormalization group (paper Sec. II.C and
 * Fig. 3): four chi x chi corners C1..C4 and four chi x chi x D^2 edge tensors
 * T1..T4 per unit-cell position, grown by directional moves and truncated to
 * chi by projectors.  It also evaluates the readouts the paper builds on that
 * environment: nearest-neighbour reduced density matrices and the energy of
 * the ruby model (Eq. H-KR, App. A), the fidelity per site (Sec. III, Eq.
 * "fidelity", Fig. 4) and the boundary density operator spectrum /
 * entanglement entropy on an infinite cylinder (Sec. IV, Eq. "rho").
 *
 * Conventions (all arrays row-major, complex values as interleaved
 * (re, im) doubles):
 *   - site tensors A[p,u,l,d,r], p physical (dimension d), u,l,d,r virtual
 *     (dimension D), unit cell Lx x Ly with x to the right and y downwards;
 *   - the double-layer tensor a[(u u'),(l l'),(d d'),(r r')], fused index
 *     ket*D + bra (Fig. 3a);
 *   - environment legs, listed so a 90-degree rotation only relabels:
 *     C1[d,r] C2[l,d] C3[u,l] C4[r,u], T1[l,d,r] T2[u,l,d] T3[r,u,l] T4[d,r,u];
 *   - a move is one direction applied to every column (row) of the cell in
 *     turn; a sweep is the moves L, R, U, D.
 *
 * Memory: the library copies the host tensors at create time; all device
 * memory of a handle comes from the caller's workspace (if given) or from
 * cudaMalloc at create time, and is released by ipeps_ctm_destroy.  Host
 * output buffers are always caller-owned.  Every call runs on the handle's
 * stream and returns when its host outputs are ready.
 *
 * Errors: every entry point returns an ipeps_status; none aborts.  On error
 * ipeps_last_error() (thread-local) holds a one-line message.  A handle stays
 * valid after an error, but its environment is unspecified after a failed
 * move.  A handle is used by one host thread at a time.
 */
#ifndef IPEPS_CTM_H
#define IPEPS_CTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipeps_ctm_s* ipeps_ctm;

typedef enum {
  IPEPS_OK = 0,
  IPEPS_EINVAL = 1,      /* bad argument (sizes, pointers, pattern)          */
  IPEPS_ENOMEM = 2,      /* device allocation or workspace too small          */
  IPEPS_ECUDA = 3,       /* a CUDA runtime call failed                        */
  IPEPS_ENOCONV = 4,     /* converge: max_sweeps reached above tolerance      */
  IPEPS_ETIMEOUT = 5,    /* an iteration budget inside a kernel ran out       */
  IPEPS_ENUMERIC = 6,    /* NaN/Inf or a zero norm met                        */
  IPEPS_EUNSUPPORTED = 7, /* option combination not built                     */
  IPEPS_EIO = 8           /* checkpoint file missing, unwritable, short, corrupt */
} ipeps_status;

typedef enum { IPEPS_REAL64 = 0, IPEPS_COMPLEX128 = 1 } ipeps_dtype;

/* Arithmetic of the contraction GEMMs.  Projector orthonormalisation (its
 * Grams FP64 or FP64-accurate on the tensor cores), normalisation and readouts
 * are FP64 in every mode; the projector-core Jacobi SVD is FP64, in the
 * TF32 / BF16 forms double-float (FP32 pairs, about 48 significand bits). */
typedef enum {
  IPEPS_PREC_FP64 = 0,   /* complex FP64 on the CUDA cores                    */
  IPEPS_PREC_TF32 = 1,   /* tcgen05 TF32 tensor cores, FP32 accumulate        */
  IPEPS_PREC_BF16X3 = 2, /* tcgen05 split-BF16 (hi*hi + hi*lo + lo*hi), FP32  */
  IPEPS_PREC_BF16X6 = 3, /* tcgen05 split-BF16 in three parts p0+p1+p2 (24   *
                          * significand bits), the six products p_i q_j with  *
                          * i + j <= 2, FP32 accumulate: FP32-class products  */
  IPEPS_PREC_FP64TC = 4  /* FP64-accurate products on tcgen05: each operand  *
                          * row split exactly into seven base-256 digit       *
                          * planes (BF16), the 28 plane pairs of weight <= 6  *
                          * summed exactly, one rounding to FP64 (after       *
                          * Ozaki, Ogita, Oishi and Rump 2012); the range     *
                          * finder's bases by shifted CholeskyQR3 (Fukaya et  *
                          * al. 2020) instead of Jacobi, cutoff and results   *
                          * as IPEPS_PREC_FP64 (to rounding)                  */
} ipeps_prec;

typedef enum {
  IPEPS_MOVE_LEFT = 0,
  IPEPS_MOVE_UP = 1,
  IPEPS_MOVE_RIGHT = 2,
  IPEPS_MOVE_DOWN = 3,
  IPEPS_SWEEP = 4        /* L, R, U, D */
} ipeps_dir;

/* Unit cell (paper Sec. II.B: a 2x2 cell of block sites; 1x1 also allowed). */
typedef struct {
  int Lx, Ly;                       /* 1 or 2 each                                 */
  int pattern[4];                   /* tensor id at (x,y) is pattern[y*Lx + x]     */
  int n_tensors;                    /* 1..4                                        */
  int d;                            /* physical dimension (8 for a block site)     */
  int D;                            /* bond dimension (a leg of size 1 is padded)  */
  ipeps_dtype dtype;                /* element type of the host tensors           */
  const void* const* tensors;       /* n_tensors host pointers, A[p,u,l,d,r]       */
  const void* const* tensors_bra;   /* NULL, or the second state B of the mixed
                                       network e = sum_p A_p conj(B_p) (Sec. III)  */
  const int* leg_dims;              /* NULL (every leg D), or 4 per tensor: the
                                       sizes (u, l, d, r), each 1 or D, of the host
                                       tensors A[p,u,l,d,r]; a leg of size 1 is a
                                       trivial bond (App. B: the empty edges of the
                                       star lattice's block sites), embedded at
                                       index 0 of a D leg                          */
} ipeps_cell;

typedef struct {
  int chi;                          /* environment bond dimension, >= D*D          */
  ipeps_prec prec;                  /* contraction arithmetic                      */
  int rsvd_oversample;              /* projector range finder width k = chi + p    */
  int rsvd_power;                   /* subspace iterations q                       */
  double svd_cutoff;                /* keep singular values > cutoff * largest;
                                       <= 0: 1e-8 (FP64, FP64TC), 1e-6 (BF16X3,
                                       BF16X6), 1e-5 (TF32)                    */
  double orth_tol;                  /* range-finder basis: drop s < tol * largest  */
  uint64_t omega_seed;              /* SplitMix64 stream of the test matrix        */
  int jacobi_max_sweeps;            /* iteration budget of every Jacobi SVD        */
  void* stream;                     /* cudaStream_t; NULL = legacy default stream  */
  void* workspace;                  /* optional caller-owned device memory         */
  size_t workspace_bytes;           /* its size; see ipeps_ctm_workspace_size      */
  long long wait_cycles;            /* limit of each device-side wait on other
                                       CTAs (the grid barrier of the small-row
                                       Jacobi), in SM clock cycles; after it the
                                       wait gives up and the call reports
                                       ETIMEOUT.  <= 0: 4e9 (about 2 s)        */
  int corners;                      /* projector of a cut (Sec. II.C): 4 (or 0)
                                       the ring of the four enlarged corners of
                                       the plaquette, X = (Q1 Q2)^T (Q4 Q3^T); 2
                                       the two corners on the cut's side,
                                       X = Q1^T Q4 (about a third of the work);
                                       else EINVAL                             */
} ipeps_options;

/* Fill *opt (caller-owned) with the defaults: prec FP64, oversample 16,
 * power 2, cutoff 0 (automatic), orth_tol 1e-14, omega_seed 7,
 * jacobi_max_sweeps 40, NULL stream/workspace, wait_cycles 0 (automatic).  chi is set to 0 and must be
 * chosen by the caller.  The projector choices are the readings of the CTM
 * the paper cites in Sec. II.C (it prints none).  No effect if opt is NULL. */
void ipeps_default_options(ipeps_options* opt);

/* Device bytes a handle with this cell/options needs, for sizing a
 * caller-owned workspace (ipeps_options.workspace).  Host only: no CUDA call.
 * *bytes is written (caller-owned).  Errors: EINVAL (the checks of
 * ipeps_ctm_create on cell and options, or bytes NULL). */
ipeps_status ipeps_ctm_workspace_size(const ipeps_cell* cell, const ipeps_options* opt,
                                      size_t* bytes);

/* Copy the tensors to the device, build every double-layer tensor (Fig. 3a;
 * the mixed e of Sec. III when tensors_bra is given), and initialise the
 * environment by tracing the outer legs of the neighbouring sites ket against
 * bra (Sec. II.C, environment of Fig. 3b).  The host tensors are copied and
 * may be freed on return; *out is a new handle owned by the caller (release
 * it with ipeps_ctm_destroy).  Errors: EINVAL (cell or options out of range:
 * Lx/Ly not in {1,2}, n_tensors not 1..4, pattern ids out of range, d not
 * 1..64, D not 1..12, chi < D*D or chi + oversample > 1024, bad dtype or
 * prec, NULL pointers), ENOMEM (device allocation failed or the caller's
 * workspace is smaller than ipeps_ctm_workspace_size), ECUDA, ENUMERIC (a
 * zero-norm initial environment tensor); *out is left unset on error. */
ipeps_status ipeps_ctm_create(const ipeps_cell* cell, const ipeps_options* opt, ipeps_ctm* out);

/* Replace the site tensors (same shapes) and rebuild the double layers; the
 * environment is kept, as when an update step reuses it (Sec. II.C).  With
 * tensors == NULL the double layers are rebuilt from the tensors already on
 * the device (no copy; the call does not wait for the device).  Host tensors
 * are copied (caller-owned).  Errors: EINVAL (NULL handle; tensors_bra given
 * or omitted unlike at create), ECUDA. */
ipeps_status ipeps_ctm_set_tensors(ipeps_ctm h, const void* const* tensors,
                                   const void* const* tensors_bra);

/* Re-run the trace initialisation of the environment (as at create).
 * Errors: EINVAL (NULL handle), ECUDA, ENUMERIC (a zero-norm tensor). */
ipeps_status ipeps_ctm_reset_env(ipeps_ctm h);

/* Apply `count` moves in direction dir (ipeps_dir).  Each move computes the
 * enlarged corners, the projectors of every cut and renormalises the
 * corners/edges of each column (row) of the cell in turn (Sec. II.C, Fig. 3b:
 * the environment is grown and truncated back to chi).  The work of one
 * move (or sweep) in a direction is captured once as a CUDA graph, on a
 * stream of the handle's own, and launched on the handle's stream for every
 * later call (one launch per move; the handle's buffers never move, so the
 * graph stays valid until ipeps_ctm_autotune changes the tile choices);
 * while kernel-class profiling is enabled the kernels are launched one by
 * one instead.  Returns when the moves are done.  Errors: EINVAL (NULL
 * handle, dir outside 0..4, count < 0),
 * ENOMEM (scratch), ECUDA, ETIMEOUT (a Jacobi SVD or a tensor-core wait ran
 * out of its budget), ENUMERIC (NaN/Inf or a zero norm); after an error the
 * environment is unspecified (ipeps_ctm_reset_env or ipeps_ctm_load restores
 * a defined one). */
ipeps_status ipeps_ctm_move(ipeps_ctm h, int dir, int count);

/* Implementation support (no paper counterpart).
 * Autotune the tensor-core products of this handle: one sweep and one bond
 * readout (the two-site RDMs) are run with every product shape timed under
 * each candidate tile choice (128 x 128 or 128 x 256 output tiles, K splits)
 * and the fastest recorded; later moves and readouts use the recorded choices
 * (results change only by rounding).  The environment and the cuts' Jacobi
 * starts are restored afterwards (a temporary device copy of them is
 * allocated for the call).  No-op for IPEPS_PREC_FP64 and IPEPS_PREC_FP64TC (their
 * digit-split products choose tiles by a cost model).  ipeps_ctm_tuning_size: number of
 * product shapes tuned.  Errors: ECUDA, ENOMEM-class CUDA failures, and any
 * status of the tuning sweep. */
ipeps_status ipeps_ctm_autotune(ipeps_ctm h);
int ipeps_ctm_tuning_size(ipeps_ctm h);

/* Singular values of every corner, divided by the largest (the corner
 * spectra whose change measures the convergence of the environment, Sec.
 * II.C): s_out is [4][Ly][Lx][chi] doubles (C1..C4), descending, zeros past
 * the rank, caller-owned host memory.  Errors: EINVAL (NULL argument), ECUDA,
 * ETIMEOUT (Jacobi budget). */
ipeps_status ipeps_ctm_spectra(ipeps_ctm h, double* s_out);

/* Sweep until max over corners of ||s/s_0 - s_old/s_old_0||_2 < tol or
 * max_sweeps is reached (Sec. II.C: moves repeated until the environment
 * converges).  *sweeps = sweeps done, *delta = the last change (caller-owned,
 * either may be NULL; both are written on ENOCONV too).  Errors: EINVAL (NULL
 * handle), ENOCONV (max_sweeps reached, or max_sweeps <= 0), and any error of
 * ipeps_ctm_move / ipeps_ctm_spectra. */
ipeps_status ipeps_ctm_converge(ipeps_ctm h, double tol, int max_sweeps, int* sweeps,
                                double* delta);

/* Nearest-neighbour two-site RDMs normalised to trace one (paper Sec. II.C,
 * used for the correlators of Sec. VI).  rho_h: bonds (x,y)-(x+1,y), rho_v:
 * bonds (x,y)-(x,y+1), each [Ly][Lx][d*d][d*d] complex (interleaved doubles),
 * rows (p_first, p_second) ket, columns the bra pair; caller-owned host
 * memory, either may be NULL.  Errors: EINVAL (NULL handle), ENOMEM
 * (scratch), ECUDA, ENUMERIC (zero trace). */
ipeps_status ipeps_rdm(ipeps_ctm h, double* rho_h, double* rho_v);

/* One-site RDMs normalised to trace one (Sec. II.C: the site's physical legs
 * left open inside its 3x3 window C1 T1 C2 / T4 . T2 / C4 T3 C3 of Fig. 3b).
 * rho_s: [Ly][Lx][d][d] complex (interleaved doubles), rows ket, columns bra,
 * caller-owned.  At a converged environment these equal the partial traces
 * of the bond RDMs up to the truncation error.  Errors: EINVAL (null
 * argument), ENOMEM (scratch), ECUDA, ENUMERIC. */
ipeps_status ipeps_rdm_site(ipeps_ctm h, double* rho_s);

/* Energy per spin of the ruby model H_R = -sum_a J_a sum s^a s^a (Eq. H-KR)
 * in the block-site form of App. A (2x2 cell, d = 8): J = {Jx, Jy, Jz}
 * (host, read only), *e_per_spin written (caller-owned): the trace of every
 * bond RDM with its bond operator, summed over the 8 bonds of the cell, / 12.
 * Errors: EINVAL (NULL argument; not a 2x2 cell of d = 8 sites), ENOMEM,
 * ECUDA, ENUMERIC. */
ipeps_status ipeps_energy(ipeps_ctm h, const double J[3], double* e_per_spin);

/* Energy per spin of a star-lattice spin model (App. B: the star lattice
 * mapped onto the same 2x2 cell of d = 8 triangle block sites, its empty edges
 * trivial bonds of dimension 1, ipeps_cell.leg_dims): Heisenberg couplings
 * J = {J_t (inside each triangle), J_e (between triangles)} on Pauli
 * matrices, H = J_t sum s.s + J_e sum s.s.  Reading of the block structure
 * (the figure is absent from the text): spins 1, 2, 3 of a triangle link to
 * its left, right and vertical neighbour; A sites (x+y even) link downwards,
 * B sites upwards, so the vertical bond with B on top is the trivial edge.
 * Energy per spin = (1/12) sum over the cell's 8 bonds.  Errors: EINVAL (NULL
 * argument, cell not 2x2 with d = 8), and those of ipeps_rdm. */
ipeps_status ipeps_energy_star(ipeps_ctm h, const double J[2], double* e_per_spin);

/* Partition-function ratio kappa = Z(window) Z(corners) / (Z(columns)
 * Z(rows)) of the 2x2 window of sites at (0,0), cell indices taken mod
 * (Lx, Ly) (Eq. "fidelity", Fig. 4): the weight of those four sites per unit
 * of infinite lattice.  kappa_out = {re, im} (2 caller-owned doubles).
 * Errors: EINVAL (NULL argument), ENOMEM, ECUDA, ENUMERIC. */
ipeps_status ipeps_kappa(ipeps_ctm h, double* kappa_out);

/* Fidelity per block site d = |k12|^(1/4) / (|k11| |k22|)^(1/8) (the 2x2 window),
 * from a converged mixed-network handle h12 (tensors_bra set) and the two
 * converged plain handles (Sec. III, Eq. "fidelity"); d_spin = d_block^(1/3).
 * Outputs are caller-owned doubles, either may be NULL.  Errors: EINVAL
 * (NULL handle; the three cells differ in Lx, Ly), and any error of
 * ipeps_kappa on the three handles. */
ipeps_status ipeps_fidelity(ipeps_ctm h12, ipeps_ctm h11, ipeps_ctm h22, double* d_block,
                            double* d_spin);

/* Boundary density operator on a cylinder of circumference Nv block sites
 * (a multiple of Ly) cut between columns x and x+1 (Sec. IV): sigma_R = ring
 * of T2 at column x, sigma_L = ring of T4 at column x+1; eigenvalues of
 * sigma_L^T sigma_R through sqrt(sigma_L^T) sigma_R sqrt(sigma_L^T) after
 * Hermitising, normalised to sum 1, descending.  eig_out holds D^Nv doubles
 * (caller-owned, may be NULL), *n_out = D^Nv, *S_vn = -sum l ln l.  EINVAL
 * if D^Nv > 4096. */
ipeps_status ipeps_boundary_rho(ipeps_ctm h, int x, int Nv, double* eig_out, int* n_out,
                                double* S_vn);

/* Boundary spectrum beyond the ring approximation (Sec. IV: sigma_L and
 * sigma_R are the dominant left and right eigenvectors of the cylinder's
 * column transfer matrix; the rings of T approximate them).  Starting from
 * the rings of ipeps_boundary_rho, power iteration with the exact transfer
 * matrix of one cell period (sigma_R <- E_{x+1} .. E_{x+Lx} sigma_R, sigma_L
 * <- sigma_L E_{x-Lx+1} .. E_x; E_c the column of double-layer tensors of
 * cell column c, periodic over Nv rows), each iterate normalised and its
 * phase aligned with the previous one, until both rings change by less than
 * tol (Frobenius) or after iters iterations; then the spectrum and entropy as
 * ipeps_boundary_rho.  *iters_used and *change report the iteration (either
 * may be NULL); eig_out holds D^Nv doubles (caller-owned, may be NULL).
 * Allocates about 9 D^(2 Nv) + 5 D^(2 Nv + 4) complex numbers for its
 * duration.  Errors: EINVAL (Nv not a multiple of Ly, iters < 0, D^Nv > 4096,
 * D^(2 Nv + 4) > 2^28), ENOMEM, ECUDA, ENUMERIC, ETIMEOUT (Jacobi budget). */
ipeps_status ipeps_boundary_rho_refined(ipeps_ctm h, int x, int Nv, int iters, double tol, double* eig_out,
                                        int* n_out, double* S_vn, int* iters_used, double* change);

/* Second Renyi entropy of the boundary density operator (Sec. IV): with
 * sigma_L, sigma_R the rings of ipeps_boundary_rho (phase-fixed, Hermitised)
 * and M = sigma_L^T sigma_R formed densely (D^Nv x D^Nv, one GEMM in the
 * handle's contraction arithmetic), *purity = Re tr(M^2) / (Re tr M)^2 =
 * sum lam^2 over the normalised spectrum and *S2 = -ln(purity); both
 * caller-owned, either may be NULL.  Needs no eigenvalues, so it is defined
 * for cylinders whose spectrum is only known in part (the leading-k route).
 * Allocates about 3 n^2 complex numbers plus the product's operands (n =
 * D^Nv; about 190 GB at D = 6, Nv = 6) for its duration.  Errors: EINVAL
 * (Nv not a multiple of Ly, D^Nv above 4096 for the FP64 path or above
 * 200000), ENOMEM (that allocation), ECUDA, ENUMERIC (a zero trace). */
ipeps_status ipeps_boundary_renyi2(ipeps_ctm h, int x, int Nv, double* S2, double* purity);

/* Leading boundary spectrum for cylinders beyond the dense route (Sec. IV:
 * for long circumferences only the leading eigenvalues of sigma_L^T sigma_R
 * are computed, iteratively).  sigma_L and sigma_R (as in ipeps_boundary_rho,
 * n = D^Nv) are built as dense n x n operators, each by one product of two
 * half rings in the handle's contraction arithmetic (tensor cores in the
 * precision forms), phase-fixed and Hermitised.  The k largest eigenvalues of
 * M = sigma_L^T sigma_R then come from a Lanczos iteration in the sigma_R
 * inner product <x,y> = x^H sigma_R y, in which M is self-adjoint when
 * sigma_R is positive definite, with full reorthogonalisation: Krylov
 * vectors, inner products, reorthogonalisation and the tridiagonal eigenvalues
 * in FP64; the mat-vec products in FP64 for an FP64 handle and on the FP32
 * pipe with FP64 accumulation in the precision forms (whose ring operators
 * carry ~1e-6 relative error).  It stops when each of the k Ritz values has
 * residual <= tol times the largest, or after max_iter steps.  The values
 * are divided by tr M.
 *   eig_out: k doubles, descending (caller-owned host; may be NULL);
 *   *n_conv: how many of the k met tol (k when an invariant subspace was hit);
 *   *S_vn = -sum lam ln lam over the k values; *rest = 1 - sum of the k.
 * Device memory: allocated for the duration of the call (about 2 n^2 +
 * chi^2 (D^Nv + 1.6 n) complex numbers for the two operators and the ring
 * product) and freed before it returns.  Errors: EINVAL (Nv not a multiple of
 * Ly or < 2, D^Nv > 200000, not 1 <= k <= max_iter <= min(1024, n), tol <= 0),
 * ENOMEM, ENUMERIC (sigma_R not positive definite: a negative norm met),
 * ETIMEOUT (Jacobi budget of the tridiagonal eigensolve). */
ipeps_status ipeps_boundary_rho_topk(ipeps_ctm h, int x, int Nv, int k, int max_iter, double tol,
                                     double* eig_out, int* n_conv, double* S_vn, double* rest);

/* Copy one environment tensor (Fig. 3b: the C and T of Sec. II.C) to the
 * host: role 0..3 = C1..C4 (chi*chi complex), 4..7 = T1..T4 (chi*D*D*chi
 * complex), at cell position (x,y); host_out is caller-owned, interleaved
 * doubles, row-major in the leg order of the conventions above.  Errors:
 * EINVAL (NULL argument, role outside 0..7, position outside the cell),
 * ECUDA. */
ipeps_status ipeps_ctm_env_get(ipeps_ctm h, int role, int x, int y, double* host_out);

/* Overwrite one environment tensor (Sec. II.C, Fig. 3b) from the host, same
 * role / position /
 * layout as ipeps_ctm_env_get (complex128, interleaved re, im; C[a,b] chi*chi
 * and T[a,k,b] chi*D*D*chi row-major, the D*D leg fused ket*D + bra).  This is
 * the user-supplied initial environment (instead of the trace initialisation
 * of create / reset_env): the next move starts from what was set.  The
 * library copies the data; nothing is normalised.  Errors: EINVAL (null
 * pointer, role outside 0..7, position outside the cell), ECUDA. */
ipeps_status ipeps_ctm_env_set(ipeps_ctm h, int role, int x, int y, const double* host_in);

/* Copy the whole environment (every C and T of the cell, Sec. II.C) of src
 * into dst on the device, e.g. from a precision-form handle into an
 * IPEPS_PREC_FP64TC or IPEPS_PREC_FP64 one to finish a convergence in FP64
 * arithmetic.  The handles must have the same Lx, Ly, D and chi (their site
 * tensors and options may differ).  Asynchronous: queued on dst's stream after
 * the work queued on src's, and src's stream waits for the copy.  No paper
 * counterpart.  Errors: EINVAL (NULL handle, different cell geometry), ECUDA. */
ipeps_status ipeps_ctm_env_copy(ipeps_ctm dst, ipeps_ctm src);

/* Checkpoint and resume of the environment (the CTM state that moves
 * update; the site tensors and options are the caller's and are not stored).
 * No paper counterpart: persistence of the state of Sec. II.C.
 *
 * File format (little-endian):
 *   bytes 0..7    "IPEPSENV"
 *   12 x int32    version (1), Lx, Ly, d, D, chi, n_tensors, pattern[4], 0
 *   payload       for site y*Lx + x in order, for role 0..7 (C1..C4, T1..T4):
 *                 the tensor as ipeps_ctm_env_get returns it (complex128)
 *   uint64        checksum of the payload: h = 0xcbf29ce484222325, then for
 *                 each 8-byte little-endian word w: h = (h ^ w) * 0x100000001b3
 *                 (mod 2^64; FNV-1a applied to 64-bit words)
 *
 * ipeps_ctm_save writes `path` through a temporary "<path>.part" renamed on
 * success, so an interrupted save leaves any earlier file intact.  Errors:
 * EINVAL (null argument), ECUDA, EIO (cannot write). */
ipeps_status ipeps_ctm_save(ipeps_ctm h, const char* path);

/* Load a checkpoint written by ipeps_ctm_save into a handle with the same Lx,
 * Ly, D and chi (d, the tensors and the pattern may differ: a converged
 * environment of one coupling point is a warm start for a nearby one).  The
 * file is read and its checksum verified before the handle is touched, so
 * after EINVAL or EIO the environment is unchanged (after ECUDA it may be
 * partly loaded).  Errors: EINVAL (null argument, geometry differs), EIO
 * (missing, short, not a checkpoint, bad checksum), ECUDA. */
ipeps_status ipeps_ctm_load(ipeps_ctm h, const char* path);

/* Read and verify a checkpoint's header and checksum without a handle or a
 * GPU (no paper counterpart; see ipeps_ctm_save).  info (caller-owned, 11 ints): version, Lx, Ly, d, D, chi, n_tensors,
 * pattern[4].  Errors: EINVAL (null argument), EIO as ipeps_ctm_load. */
ipeps_status ipeps_env_file_info(const char* path, int* info);

/* Block until all work of the handle is done (no paper counterpart).
 * Errors: EINVAL (NULL handle), ECUDA (an earlier asynchronous failure). */
ipeps_status ipeps_ctm_sync(ipeps_ctm h);

/* Number of kernels this handle launched since create (a counter kept on
 * the host, for launch accounting; no paper counterpart).  0 for NULL. */
uint64_t ipeps_ctm_launch_count(ipeps_ctm h);

/* Kernel-class timing for roofline reports: with enable != 0 every
 * contraction GEMM (kind 0), every Jacobi SVD (kind 1) and every FP64 GEMM of
 * the precision form's projector step (kind 2: CholeskyQR Grams and applies,
 * core products) is bracketed by CUDA events on the stream that runs it.
 * profile() clears the records; profile_read() synchronises and returns the
 * summed event time (ms), the number of launches and (kinds 0, 2) the
 * algorithmic flops (8*M*N*K per complex GEMM; Hermitian and triangular
 * results count their nonzero part), or (kind 1) the mean number of sweeps per
 * Jacobi call.  ipeps_boundary_rho_topk adds kind 3 (building both dense ring
 * operators; flops: the two ring products, 16 n^2 chi^2) and kind 4 (the
 * Lanczos iteration; "flops" holds its step count).  Tensor-core products
 * are also timed without their operand packing: kind 5 the main tcgen05
 * kernel of products with more than 256 output rows (enlarged corners,
 * absorption, readouts) and kind 6 of thin products (at most 256 rows: the
 * range finder and the projector assembly), each with algorithmic flops;
 * kind 7 the kind-6 launches again with the bytes the kernel must move
 * (packed operands read once, output or FP32 partials written once) in the
 * third output; kind 8 the split-K reductions with their bytes.  With two
 * projector lanes the brackets of concurrent work overlap, so class times can
 * sum to more than the step.  While enabled, moves run without CUDA graphs
 * (the events are per launch).  Not a paper
 * operation: measurement support only.  The outputs of profile_read are
 * caller-owned and may each be NULL.  Errors: EINVAL (NULL handle), ECUDA. */
ipeps_status ipeps_ctm_profile(ipeps_ctm h, int enable);
ipeps_status ipeps_ctm_profile_read(ipeps_ctm h, int kind, double* total_ms, uint64_t* launches,
                                    double* flops);

/* Wait for the handle's work, then release everything it allocated (a
 * caller's workspace stays the caller's).  NULL is a no-op. */
void ipeps_ctm_destroy(ipeps_ctm h);

/* Building block, no paper counterpart.
 * Complex GEMM building block of every contraction, for unit tests: C = opA(A)
 * opB(B) with M x N output, complex interleaved doubles in host memory
 * (row-major; op 0 = N, 1 = T, 2 = conj, 3 = conj-transpose, so that opA(A)
 * is M x K and A is stored M x K for op 0/2 and K x M for op 1/3).  prec as
 * ipeps_prec: FP64 CUDA-core kernel or the tcgen05 TF32 / split-BF16x3 /
 * split-BF16x6 kernel, or IPEPS_PREC_FP64TC: the FP64-accurate tensor-core
 * product (exact base-256 digit splitting of both operands, digit-plane
 * products summed exactly; the one rounding to FP64 is the last)
 * (with its operand packing and split-K reduction).  Allocates and frees its
 * own device buffers; synchronises the device.  A, B, C are caller-owned host
 * arrays.  Errors: EINVAL (M, N or K <= 0, NULL pointer, prec or op out of
 * range), ECUDA (including a failed device allocation), ETIMEOUT (a
 * tensor-core wait ran out). */
ipeps_status ipeps_zgemm(int prec, int M, int N, int K, const double* A, int opA, const double* B, int opB,
                         double* C);

/* As ipeps_zgemm for the tensor-core precisions, with the tile choice fixed
 * instead of the default: output tiles of 128 x bn real columns (bn = 128 or
 * 256; 256 applies where 2N padded to 128 is a multiple of 256, else 128
 * is used) and `splits` K splits (reduced to the number of k-blocks, 128 bytes
 * of K, 64 for BF16X6, if larger).  For unit tests of every choice the
 * batch autotuner can make (no paper counterpart).  Host buffers as
 * ipeps_zgemm.  Errors: EINVAL (prec FP64, bn not 128 or 256, splits < 1, or
 * as ipeps_zgemm), ECUDA, ETIMEOUT. */
ipeps_status ipeps_zgemm_tile(int prec, int bn, int splits, int M, int N, int K, const double* A, int opA,
                              const double* B, int opB, double* C);

/* Corner spectrum without any device allocation (the paper has no
 * counterpart: this is an interface for callers that cannot call cudaMalloc,
 * e.g. a process whose device memory is owned entirely by another allocator,
 * or a loop that must not take the device synchronisation of cudaMalloc /
 * cudaFree).  C_dev: device pointer to one chi x chi complex corner matrix
 * (interleaved doubles, row-major, read only); s_dev: device pointer to chi
 * doubles receiving its singular values in descending order divided by the
 * largest (zeros where the matrix has none) -- the same values
 * ipeps_ctm_spectra returns for a corner.  stream: cudaStream_t (NULL =
 * default stream); the call synchronises that stream (it reads the SVD's
 * status back) and returns when s_dev is written.
 * All intermediates live in one fixed device array of about 1 MiB inside
 * the library (every GPU that loads the library holds it until exit), so
 * chi is limited to 1..256; larger chi returns EINVAL.  Every call looks up
 * that array's device address with the caller's device current; the first
 * call on a device also loads the library's device code there.  All calls
 * share the array: two
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and give wrong results.  Errors: EINVAL (null pointer, chi out of range),
 * ECUDA, ETIMEOUT (Jacobi sweep budget), with ipeps_last_error(). */
ipeps_status ipeps_corner_spectrum_noalloc(const double* C_dev, int chi, double* s_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Batched scan: n independent instances (e.g. the coupling points of a
 * phase-diagram scan, Sec. VI, each with its own tensors, D and chi) advanced
 * together.  Each instance is an ordinary handle with its own device memory
 * (allocated at create) and its own stream; a batch move is captured once per
 * direction as one CUDA graph with one branch per instance and replayed, so
 * one graph launch advances every instance and the GPU overlaps their small
 * contractions.  Tensor-core products take the tile shape (128 x 128 or
 * 128 x 256 output tiles) and K-split count chosen per product shape by the
 * library's autotuner.
 * ------------------------------------------------------------------------- */
typedef struct ipeps_batch_s* ipeps_batch;

/* Create the n instances: cells[i], opts[i] as for ipeps_ctm_create (the
 * stream and workspace fields are ignored: the batch owns one stream per
 * instance and each instance allocates its own memory).  With tune != 0 the
 * autotuner times every candidate tile choice of every distinct tensor-core
 * product shape during one sweep of each instance (cuts in sequence), after
 * which each environment is re-initialised by the trace initialisation; with
 * tune == 0 the default choice applies.  Errors: as ipeps_ctm_create, with
 * the failing instance named in ipeps_last_error(); nothing is left allocated
 * on error. */
ipeps_status ipeps_batch_create(int n, const ipeps_cell* cells, const ipeps_options* opts, int tune,
                                ipeps_batch* out);

/* `count` moves (ipeps_dir, IPEPS_SWEEP = L, R, U, D) of every instance.  The
 * first call per direction captures the graph; every call replays it `count`
 * times and returns when all instances are done.  Each instance computes
 * exactly what ipeps_ctm_move computes on it.  Errors: the first failing
 * instance's status (ETIMEOUT, ENUMERIC, ...), named in ipeps_last_error(). */
ipeps_status ipeps_batch_move(ipeps_batch b, int dir, int count);

/* Energy per spin of every instance (as ipeps_energy, Eq. H-KR), J = n x
 * {Jx, Jy, Jz}, e_out = n doubles; both caller-owned host arrays.  Errors:
 * EINVAL (NULL argument), or the first failing instance's ipeps_energy
 * status. */
ipeps_status ipeps_batch_energy(ipeps_batch b, const double* J, double* e_out);

/* Fidelity surface (Sec. VI: the fidelity per site of the states at two
 * coupling points J1, J2 of a parameter line, Sec. III, Eq. "fidelity"): for
 * each of the n_pairs pairs p, i12[p] is the batch instance holding the mixed
 * network of the two states (created with tensors_bra), i11[p] and i22[p] the
 * instances of the two plain networks, all with the same Lx, Ly; d_block[p]
 * and (if d_spin is not NULL) d_spin[p] receive the fidelity per block site
 * and per spin exactly as ipeps_fidelity computes them.  The kappa of every
 * instance the pairs name is computed once.  Index arrays and outputs are
 * caller-owned host arrays of n_pairs entries.  Errors: EINVAL (NULL batch or
 * array, an index out of range, cells that differ within a pair), or the
 * first failing instance's ipeps_kappa status, named in ipeps_last_error(). */
ipeps_status ipeps_batch_fidelity(ipeps_batch b, int n_pairs, const int* i12, const int* i11, const int* i22,
                                  double* d_block, double* d_spin);

/* Instance i as a handle for every single-instance readout (spectra, RDMs,
 * kappa, boundary rho, env_get).  Owned by the batch: do not destroy it; do
 * not move it while a batch move of the same batch is in flight.  NULL if i is
 * out of range. */
ipeps_ctm ipeps_batch_instance(ipeps_batch b, int i);

/* Autotuner table (implementation support, no paper counterpart): number of
 * product shapes tuned (0 for NULL), and entry i as fields = {prec, M, N, K,
 * n-tile width, K splits} (M x N x K the complex product) and us = {time of
 * the chosen tile, time of the default choice} in microseconds, both
 * caller-owned.  Errors: EINVAL (NULL argument, i out of range). */
int ipeps_batch_tuning_size(ipeps_batch b);
ipeps_status ipeps_batch_tuning_entry(ipeps_batch b, int i, int fields[6], double us[2]);

/* Kernels the batch launched since create (graph replays count every kernel
 * inside the graph; launch accounting, no paper counterpart).  0 for NULL. */
uint64_t ipeps_batch_launch_count(ipeps_batch b);

/* Block until all work of the batch is done.  Errors: EINVAL (NULL batch),
 * ECUDA. */
ipeps_status ipeps_batch_sync(ipeps_batch b);

/* The batch's own stream (cudaStream_t, owned by the batch): the graph of
 * every batch move is launched on it, so events recorded on it before and
 * after ipeps_batch_move bracket the whole move on the device.  NULL for a
 * NULL batch. */
void* ipeps_batch_stream(ipeps_batch b);

/* Wait for the batch's work, then release its graphs, streams, tuner and
 * every instance handle.  NULL is a no-op. */
void ipeps_batch_destroy(ipeps_batch b);

/* Thread-local message of the last failed call on this thread ("" if none);
 * owned by the library, valid until the next failing call on this thread. */
const char* ipeps_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IPEPS_CTM_H */
