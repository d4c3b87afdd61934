/*
 * omen.h — C ABI of the GB300 tight-binding / Schrödinger–Poisson library.
 *
 * The calls follow the problem statement of OMEN 3-D (Lee, Ryu, Jiang, Klimeck,
 * "Million Atom Electronic Structure and Device Calculations on Peta-Scale Computers"):
 * an atomistic zincblende structure (Section I, Section II-A) → an empirical sp3s* /
 * sp3d5s* tight-binding Hamiltonian with strain (Section I, abstract) → its eigenstates
 * by an iterative (block) Lanczos solver (Section III-A item 1; benchmark unit "500 Lanczos
 * iterations", Section II-B) → charge (Section III-A item 2) → finite-difference Poisson
 * (Section III-A item 3) → self-consistent loop (Section III-A).
 *
 * Conventions (all calls):
 *  - Every call returns an omen_status; nothing aborts or traps.  After a failure,
 *    omen_last_error(ctx) returns a message (valid until the next call on ctx).
 *  - Pointers named *_dev are device pointers on ctx's device; work is issued on ctx's
 *    stream.  Pointers named *_host are host memory.  Caller owns every buffer it passes;
 *    the library owns the opaque handles (free with the matching omen_free_*).
 *  - One ctx per host thread.  Units: eV, nm, V, C/m^3, 1/nm.
 *  - Structure layout: conventional cubic cells, cell = (iz*ny + iy)*nx + ix; 8 sites per
 *    cell, site b in 0..3 on the first FCC sublattice (A) at a/4*(0,0,0),(0,2,2),(2,0,2),
 *    (2,2,0), b in 4..7 on the second (B) at the A site + a/4*(1,1,1).
 *    atom = b*ncells + cell.
 *  - Bond slots: A site s of cell c along direction k (a/4 units: k=0 (1,1,1), 1 (1,-1,-1),
 *    2 (-1,1,-1), 3 (-1,-1,1), pointing from the A atom to the B atom):
 *    slot = (k*4 + s)*ncells + c.
 *  - Vector layout (H rows): row = o*natoms + atom, o = spin*norb + orbital; orbitals
 *    s, px, py, pz, [dyz, dzx, dxy, dx2-y2, d3z2-r2], s*.  A block of nvec vectors is
 *    stored vector after vector ([nvec][nrows]).  Real Hamiltonians use double (F64) or
 *    float (F32) elements; complex ones (spin-orbit or Bloch phase) interleave re,im.
 */
#ifndef OMEN_H
#define OMEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OMEN_OK = 0,
  OMEN_EINVAL = 1,       /* bad argument (message says which) */
  OMEN_ENOMEM = 2,       /* device or host allocation failed */
  OMEN_ENOCONV = 3,      /* iteration limit reached; partial results and info are filled */
  OMEN_ENUMERIC = 4,     /* NaN/Inf or breakdown that could not be recovered */
  OMEN_ETIMEOUT = 5,     /* reserved: no kernel of this build waits on a flag (the CG solver's
                            grid barriers are those of a cooperative launch) */
  OMEN_ECUDA = 6,        /* CUDA runtime error (message has the CUDA error string) */
  OMEN_EUNSUPPORTED = 7  /* valid request that this build does not implement */
} omen_status;

enum { OMEN_SP3S = 5, OMEN_SP3D5S = 10 };                   /* orbitals per atom and spin */
enum { OMEN_HARD_WALL = 0, OMEN_PERIODIC = 1, OMEN_BLOCH = 2 }; /* per-direction boundary */
enum {
  OMEN_F64 = 0,          /* FP64 storage and arithmetic */
  OMEN_F32 = 1,          /* FP32 bond blocks and Krylov vectors (complex64 when complex);
                            Lanczos dots, orthogonalisation coefficients and the projected
                            eigenproblem in FP64 */
  OMEN_F32_REFINE64 = 2, /* OMEN_F32 solve, then an FP64 Rayleigh–Ritz refinement inside
                            omen_eigs; the vectors of omen_hx, omen_hx_host and v0 are FP32
                            (complex64), the eigenvectors omen_eigs returns are FP64 */
  OMEN_F64_DF = 3        /* FP64-accurate H·X on the FP32 pipe: blocks and vectors stored as
                            double-float pairs (hi, lo) of FP32 (value = hi + lo, about 48
                            significant bits), products and sums with error-free
                            transformations (Dekker 1971; Knuth TwoSum).  Real Hamiltonians
                            only; omen_hx / omen_hx_kbatch vectors are float2 (hi, lo) per
                            element (see omen_convert_vectors); omen_hx_host takes FP64. */
};
enum { OMEN_LOWEST = 0, OMEN_NEAREST = 1, OMEN_HIGHEST = 2 };  /* which eigenvalues */

typedef struct omen_ctx omen_ctx;
typedef struct omen_lattice omen_lattice;
typedef struct omen_ham omen_ham;

/* ---- context --------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`, issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Allocates small device work buffers. */
omen_status omen_create(omen_ctx** out, int device, void* cuda_stream);
void omen_destroy(omen_ctx* ctx);
const char* omen_last_error(const omen_ctx* ctx);

/* Replay Lanczos steps as CUDA graphs (default on).  The single-vector solver captures the
 * kernel sequence of the steps between two host convergence checks once and replays it on
 * later cycles; results are identical either way (same kernels, same order).  The paper has
 * no counterpart: launch overhead was not a cost on its CPUs.  EINVAL for a null context. */
omen_status omen_set_graph_capture(omen_ctx* ctx, int enable);

/* Orthogonalisation of the single-vector Lanczos steps.  Every step removes the new vector's
 * components along v_j and v_{j-1} (three-term recurrence) and measures its overlaps h with the
 * whole basis (a projection pass).  OMEN_REORTH_FULL (default) subtracts V h at every step.
 * OMEN_REORTH_SEMI subtracts it only when some |h_i| exceeds sqrt(u) ||w|| (u the vectors' unit
 * roundoff) or the previous step did so, which keeps the basis semi-orthogonal — enough for
 * Ritz values of working accuracy (Simon, Math. Comp. 42 (1984) 115; the paper's Lanczos
 * solver, Section III-A item 1, does not say how it orthogonalises).  It saves the update only
 * while no Ritz pair has converged; it costs one extra norm per step.  The first step after a
 * start or restart always takes two full passes.  OMEN_REORTH_PARTIAL (FP64 vectors, real or
 * complex; other vectors keep the full pass) skips the projection as well: it estimates the
 * overlaps of each new vector with the basis from the projected matrix by Simon's recurrence
 * (omega_{j+1} from omega_j, omega_{j-1}, the columns of T and a rounding term; the estimate
 * recurrence as in Larsen's PROPACK) and runs the full pass, for that vector and the next, only
 * when an estimate exceeds the square root of the unit roundoff.  A step then reads the basis only
 * when a pass runs.  The estimates do not follow the overlaps that the Ritz vectors kept at a
 * thick restart carry from one cycle to the next: OMEN_LOWEST solves through many restarts can
 * stall (ENOCONV; a stop is confirmed by FP64 residuals on H first), so the policy suits fixed
 * step counts and folded solves.  Every result is checked by FP64 residuals.  EINVAL for another
 * value. */
enum { OMEN_REORTH_FULL = 0, OMEN_REORTH_SEMI = 1, OMEN_REORTH_PARTIAL = 2 };
omen_status omen_set_reorthogonalization(omen_ctx* ctx, int policy);

/* Missed-copy check of single-vector solves for the lowest eigenvalues (default on).  A
 * single-vector Krylov space holds one direction of each eigenspace, so of a degenerate level
 * (symmetric structures, zone-boundary bands) it finds one copy and may report the next
 * eigenvalue in place of the others.  With the check, omen_eigs (block 1) and
 * omen_eigs_kbatch[_multi] (OMEN_LOWEST or OMEN_NEAREST) solve again for the extreme
 * eigenvalue of their operator (H, or (H - sigma)^2 for NEAREST) with the nev vectors found
 * projected out (locking); a level nearer the target than the farthest one found, by more than
 * tol, is inserted in order and the check repeats.  A block solve with block >= the
 * multiplicity needs no check. */
omen_status omen_set_locking_check(omen_ctx* ctx, int enable);

/* The device's FP64 fused multiply-add rate in TFLOP/s (no counterpart in the paper): eight
 * independent FMA chains per thread in one resident wave, best of three timed launches.  The FP64
 * products of this library are bound by that rate, so their roofline is reported against it. */
omen_status omen_probe_fp64_rate(omen_ctx* ctx, double* tflops);

/* ---- structure (paper Section II-A: atoms of the domain and their neighbours) ---------- */

typedef struct {
  int nx, ny, nz;            /* conventional cells along x, y, z (each >= 1) */
  int periodic[3];           /* OMEN_HARD_WALL (bonds leaving the block are dropped),
                                OMEN_PERIODIC, or OMEN_BLOCH (periodic with a Bloch phase) */
  double a_nm;               /* lattice constant (nm) */
  const uint8_t* species_host; /* [8*ncells] species index per atom (< nspecies of the
                                  parameters used with this structure) */
  const double* strain_host; /* [16*ncells] relative bond-length change per bond slot
                                (d = d0 (1 + strain)), or NULL for none; slots of bonds that
                                do not exist are ignored */
} omen_lattice_desc;

/* Copy the structure to the device.  Neighbours are implicit (computed from the cell
 * index); no neighbour list is stored.  Errors: EINVAL (sizes), ENOMEM. */
omen_status omen_build_lattice(omen_ctx* ctx, const omen_lattice_desc* desc, omen_lattice** out);
void omen_free_lattice(omen_lattice* lat);
/* Number of atoms and of existing bonds (after the hard-wall rule). */
omen_status omen_lattice_counts(const omen_lattice* lat, long long* natoms, long long* nbonds);

/* Replace the structure's bond strains (relative bond-length change per bond slot, device,
 * [16*ncells], slot layout as above; slots of absent bonds are ignored), e.g. with the relaxed
 * strains of omen_relax_vff.  Hamiltonians assembled afterwards use them; Hamiltonians already
 * assembled (stored or matrix-free) keep the strain they were assembled with.  Asynchronous on
 * ctx's stream. */
omen_status omen_lattice_set_strain(omen_ctx* ctx, omen_lattice* lat, const double* strain_dev);

/* ---- valence-force-field strain relaxation (paper Section II-B: atomistic VFF strain before
 * the electronic structure; Fig. 4 benchmarks it) ------------------------------------------- */
/* Keating's form (Phys. Rev. 145, 637 (1966)), per bond b and per pair of bonds p, q at an atom:
 *   E = sum_b 3 alpha_b/(8 d_b^2) (r_b.r_b - d_b^2)^2
 *     + sum_atoms sum_{p<q} 3 beta_pq/(8 d_p d_q) (r_p.r_q + d_p d_q/3)^2,
 * r_p the vector from the atom to its neighbour along bond p, d_b = sqrt(3)/4 times the mean
 * natural lattice constant of the bond's two species, alpha_b (beta_b) the mean of the two
 * species' constants, beta_pq the mean of beta_p and beta_q.  Positions are F x0 + u: x0 the
 * ideal sites at the structure's a_nm, F a homogeneous box deformation (periodic images move
 * with it), u the displacements.  Bonds leaving a hard wall are absent (free surface).
 * u and forces are [3][natoms] device arrays: the x components of all atoms, then y, then z (nm,
 * eV/nm).  Species indices are the structure's.  Units: nm, eV; alpha, beta in eV/nm^2. */
typedef struct {
  int nspecies;              /* 1..4 */
  double a_nm[4];            /* natural lattice constant per species (nm) */
  double alpha[4];           /* bond-stretching constant per species (eV/nm^2) */
  double beta[4];            /* bond-bending constant per species (eV/nm^2) */
} omen_vff_params;

typedef struct {
  double gtol;               /* stop when every force component is below gtol (eV/nm) */
  int max_iter;              /* maximum conjugate-gradient iterations */
} omen_vff_opts;

typedef struct {
  int iterations;
  int converged;
  double energy_start, energy;  /* eV, before and after */
  double max_force;          /* max |force component| at exit (eV/nm) */
  double seconds;
} omen_vff_info;

/* Energy (E_host, may be NULL) and forces -dE/du (force_dev [3][natoms], may be NULL) at
 * displacements u_dev; F_host [9] row-major, NULL = identity.  Synchronous.  EINVAL for bad
 * parameters (nspecies, a_nm <= 0, negative constants). */
omen_status omen_vff_energy_forces(omen_ctx* ctx, const omen_lattice* lat, const omen_vff_params* p,
                                   const double* F_host, const double* u_dev, double* E_host, double* force_dev);

/* Relax u_dev (start in, relaxed displacements out) at fixed F by nonlinear conjugate gradients
 * (Polak–Ribiere, clipped at zero) with an exact line search: along a direction every Keating
 * term is the square of a quadratic in the step, so the energy is a quartic whose minimum is
 * found from its derivative's coefficients (accumulated term by term, no energy differences).
 * strain_dev (or NULL) receives |r_b|/d_b - 1 per bond slot ([16*ncells], absent bonds 0), the
 * input of omen_lattice_set_strain.  Allocates its work vectors (9 doubles per atom) on ctx's
 * stream; synchronous.  ENOCONV (u and strain still written) at max_iter, ENUMERIC on a
 * non-finite force. */
omen_status omen_relax_vff(omen_ctx* ctx, const omen_lattice* lat, const omen_vff_params* p, const double* F_host,
                           const omen_vff_opts* opts, double* u_dev, double* strain_dev, omen_vff_info* info);

/* ---- Hamiltonian (paper Section I: empirical sp3s* and sp3d5s* tight binding with strain) - */

typedef struct {
  int basis;                 /* OMEN_SP3S or OMEN_SP3D5S */
  int nspecies;              /* 1..4 */
  double onsite[4][4];       /* [species][E_s, E_p, E_d, E_s*] (eV) */
  double V[4][4][14];        /* [species of atom 1][species of atom 2][integral] (eV) at d0:
                                ss_sigma, s*s*_sigma, ss*_sigma, sp_sigma, s*p_sigma, sd_sigma,
                                s*d_sigma, pp_sigma, pp_pi, pd_sigma, pd_pi, dd_sigma, dd_pi,
                                dd_delta; the first-named orbital sits on atom 1 */
  double lambda_so[4];       /* spin-orbit lambda per species (eV): lambda L.sigma on p */
  double eta;                /* Harrison exponent: integrals scale as (d0/d)^eta */
} omen_tb_params;

typedef struct {
  int spin_orbit;            /* 0/1: double the basis and add lambda L.sigma on p */
  int precision;             /* OMEN_F64, OMEN_F32 or OMEN_F32_REFINE64 */
  int matrix_free;           /* 0: store every bond block; 1: regenerate blocks in H·X from
                                the species pair, the direction and a per-bond factor
                                (d0/d)^eta taken from the structure's strain at assembly */
  const double* k;           /* NULL or [3] Bloch wave vector (1/nm) for OMEN_BLOCH axes */
  const double* U_atom_dev;  /* NULL or [natoms] onsite potential energy (eV), e.g. -phi */
} omen_ham_opts;

/* Assemble H on the device: onsite energies (+U, + spin-orbit), Slater–Koster bond blocks
 * for the bond directions, scaled by (d0/d)^eta (Slater & Koster 1954, Table I; Harrison).
 * The structure must outlive the Hamiltonian.  Errors: EINVAL, ENOMEM, ECUDA. */
omen_status omen_assemble_H(omen_ctx* ctx, const omen_lattice* lat, const omen_tb_params* p,
                            const omen_ham_opts* opts, omen_ham** out);
void omen_free_ham(omen_ham* ham);
/* Rows of H, whether it is complex, and the element size in bytes of its vectors. */
omen_status omen_ham_shape(const omen_ham* ham, long long* nrows, int* is_complex, int* elem_bytes);
/* Replace the onsite potential (eV per atom, or per grid point of an effective-mass
 * Hamiltonian; device) without rebuilding bonds. */
omen_status omen_ham_set_potential(omen_ctx* ctx, omen_ham* ham, const double* U_atom_dev);

/* ---- effective-mass Hamiltonian (paper Section III-A item 1: the Schrödinger solver takes
 * either the tight-binding or an effective-mass Hamiltonian) ------------------------------ */

typedef struct {
  int nx, ny, nz;            /* grid points along x, y, z (each >= 1, fewer than 2^30 in all) */
  double h_nm[3];            /* grid spacings (nm) */
  double m_rel[3];           /* diagonal effective masses m_d / m0 */
  int periodic[3];           /* OMEN_HARD_WALL (psi = 0 one spacing past the end points),
                                OMEN_PERIODIC, or OMEN_BLOCH: psi(r + L_d e_d) =
                                exp(i k_d L_d) psi(r), L_d = n_d h_d (complex vectors) */
  double ec_eV;              /* band edge E_c (eV) */
  double k[3];               /* Bloch wave vector (1/nm), used on OMEN_BLOCH axes */
  int precision;             /* OMEN_F64, OMEN_F32 or OMEN_F32_REFINE64 (EUNSUPPORTED for
                                OMEN_F64_DF) */
} omen_effmass_desc;

/* Single-band effective-mass Hamiltonian with a constant diagonal mass tensor, discretised by
 * second-order central differences:
 *   (H psi)_i = (E_c + U_i + 2 sum_d t_d) psi_i - sum_d t_d (psi_{i+e_d} + psi_{i-e_d}),
 *   t_d = hbar^2 / (2 m0 m_d h_d^2).
 * Row index i = (iz*ny + iy)*nx + ix.  U_dev: NULL or [nx*ny*nz] potential energy per point
 * (eV, device, copied).  The result is an omen_ham: omen_hx, omen_hx_host, omen_eigs (all
 * orderings and block sizes), omen_density_accum (one value per point) and
 * omen_ham_set_potential (one value per point) take it; the k-batch and launch-shape calls
 * return EUNSUPPORTED.  Errors: EINVAL (sizes, spacings, masses, flags), EUNSUPPORTED,
 * ENOMEM. */
omen_status omen_assemble_effmass(omen_ctx* ctx, const omen_effmass_desc* desc, const double* U_dev,
                                  omen_ham** out);

/* y = (H - sigma) x for nvec vectors in the Hamiltonian's vector type (device).
 * x and y must not overlap.  This is the operation the Lanczos recurrence repeats. */
omen_status omen_hx(omen_ctx* ctx, const omen_ham* ham, const void* x_dev, void* y_dev,
                    int nvec, double sigma);
/* Convert n vector elements between OMEN_F64 (double) and OMEN_F64_DF (float2 hi, lo) on the
 * device (either direction; src and dst must not overlap). */
omen_status omen_convert_vectors(omen_ctx* ctx, const void* src_dev, int src_precision, void* dst_dev,
                                 int dst_precision, long long n);

/* The same product with host buffers; synchronous.  The copies overlap the product: z-slabs of
 * x go up on one copy stream while earlier slabs compute on the ctx stream and their rows of y go
 * down on another (pinned host memory makes the copies asynchronous).  The device buffers and
 * events are kept in the context between calls. */
omen_status omen_hx_host(omen_ctx* ctx, const omen_ham* ham, const void* x_host, void* y_host,
                         int nvec, double sigma);

/* ---- launch-shape tuning of the products (no counterpart in the paper) ------------------ */

typedef struct {
  int threads;               /* CTA width chosen (threads per block) */
  int rows_per_batch;        /* block rows per register batch (omen_tune_hx) or wave vectors
                                per thread (omen_tune_hx_kbatch); 0 = the built-in rule */
  int candidates;            /* launch shapes timed */
  double ms_best;            /* mean launch time of the chosen shape (ms) */
  double ms_default;         /* mean launch time of the built-in shape (ms) */
} omen_tune_result;

/* Time every compiled launch shape of omen_hx on this Hamiltonian (nvec vectors of precision
 * OMEN_F64 or OMEN_F32, `reps` timed launches each after two warm-ups, CUDA events on the ctx
 * stream) and keep the fastest for later products and solves with that vector precision.
 * Allocates and frees two scratch blocks of nvec vectors; synchronises the stream.  Results
 * of the product do not depend on the shape.  out may be NULL.  EINVAL for a precision
 * without blocks in this Hamiltonian. */
omen_status omen_tune_hx(omen_ctx* ctx, omen_ham* ham, int vec_precision, int nvec, int reps,
                         omen_tune_result* out);

/* The same for the k-batched product with nk wave vectors (Bloch Hamiltonian, stored blocks,
 * no spin-orbit); the vector precision is the Hamiltonian's. */
omen_status omen_tune_hx_kbatch(omen_ctx* ctx, omen_ham* ham, int nk, int reps, omen_tune_result* out);

/* Set a launch shape directly: threads a multiple of 32 in 32..128 (0 = default 128) and
 * rows_per_batch from the compiled set (FP32 stored blocks 1, 2, 5, and 10 without spin-orbit
 * for sp3d5s*; FP64 stored 1, 2; matrix-free 1, 2; 0 = the built-in rule; rows_per_batch must
 * divide the orbital count).  k batch: wave vectors per thread 1, 2 (FP64 and FP32) or 4 (FP32), 0 =
 * default 2.  EINVAL for a shape that is not compiled. */
omen_status omen_hx_set_tile(omen_ctx* ctx, omen_ham* ham, int vec_precision, int threads, int rows_per_batch);
omen_status omen_hx_kbatch_set_tile(omen_ctx* ctx, omen_ham* ham, int vec_precision, int threads,
                                    int k_per_thread);

/* ---- eigenpairs (paper Section III-A item 1: (block) Lanczos) -------------------------- */

typedef struct {
  int nev;                   /* wanted eigenpairs (>= 1) */
  int which;                 /* OMEN_LOWEST, OMEN_HIGHEST (Lanczos on -H), or OMEN_NEAREST
                                (folded spectrum: Lanczos on (H - sigma)^2, eigenvalues by
                                Rayleigh quotients on H) */
  double sigma;              /* shift for OMEN_NEAREST (eV) */
  double tol;                /* target bound on each eigenvalue's error (eV), from its FP64
                                residual r: min(r, r^2/gap) (Weyl / Kato–Temple) */
  int max_iter;              /* maximum block steps */
  int block;                 /* block size b (>= largest multiplicity among wanted values) */
  int basis;                 /* maximum basis size m (a multiple of b, > nev + b) */
  const void* v0_host;       /* [block][nrows] start block in the vector type of the
                                Hamiltonian's precision (FP64 for OMEN_F64_DF), or NULL for a
                                fixed default */
  const void* v0_dev;        /* the same on the device (takes precedence over v0_host), e.g.
                                a combination of the previous solve's eigenvectors */
} omen_eig_opts;

typedef struct {
  int iterations;            /* block steps taken */
  long long hx_count;        /* single-vector H·X products */
  int restarts;
  int converged;             /* 1 if every returned pair met tol */
  double max_residual;       /* max FP64 ||H x - lambda x|| over returned pairs (eV) */
  double max_error_bound;    /* max FP64 min(r, r^2/gap) over returned pairs (eV) */
  double max_residual_raw;   /* F32_REFINE64: same as max_residual before refinement */
  double seconds;            /* wall time of the call */
} omen_eig_info;

/* nev eigenpairs of H by thick-restart block Lanczos with full (twice-applied classical
 * Gram–Schmidt) reorthogonalisation.  evals_host[nev] ascending; evecs_dev (or NULL)
 * receives [nev][nrows] FP64-precision vectors (double / complex128) for OMEN_F64,
 * OMEN_F32_REFINE64 and OMEN_F64_DF, float / complex64 for OMEN_F32.  With an OMEN_F64_DF
 * Hamiltonian (block 1 only; EUNSUPPORTED otherwise) the Krylov vectors are double-float pairs
 * and every product, projection and update runs on the FP32 pipe at about 48-bit accuracy;
 * v0 is given in FP64.  Returns ENOCONV with the best current pairs if max_iter is reached. */
omen_status omen_eigs(omen_ctx* ctx, const omen_ham* ham, const omen_eig_opts* opts,
                      double* evals_host, void* evecs_dev, omen_eig_info* info);

/* ---- k batching (paper Section II-C: k-space grouping) ---------------------------------- */

/* y_k = (H(k) - sigma) x_k for nk Bloch wave vectors k_host [nk][3] (1/nm) in one launch; the
 * Hamiltonian's bond blocks (stored, no spin-orbit, Bloch-periodic structure) are shared by
 * all k, only the phase on bonds that wrap a Bloch face differs.  x_dev, y_dev: [nk][nrows]
 * complex vectors of the Hamiltonian's precision. */
omen_status omen_hx_kbatch(omen_ctx* ctx, const omen_ham* ham, int nk, const double* k_host,
                           const void* x_dev, void* y_dev, double sigma);

/* Several structures in one k batch (paper Section III-A item 1: eigenstates on finite
 * k-points; structures of different sizes batched together).  Item i: a Bloch Hamiltonian with
 * stored blocks and no spin-orbit, all items of one precision and basis, and its nk wave
 * vectors k_host [nk][3] (1/nm).  At most 16 items. */
typedef struct {
  const omen_ham* ham;
  int nk;
  const double* k_host;
} omen_kbatch_item;

/* y = (H_i(k) - sigma) x for every wave vector of every item in ONE launch over the
 * (structure, k) work list.  x_dev, y_dev: the items' [nk_i][nrows_i] complex blocks stored one
 * after another in item order.  Launch shape from the first item (omen_hx_kbatch_set_tile). */
omen_status omen_hx_kbatch_multi(omen_ctx* ctx, int nitems, const omen_kbatch_item* items,
                                 const void* x_dev, void* y_dev, double sigma);

/* nev eigenpairs for each of nk wave vectors, all solved in lockstep (single-vector thick-
 * restart Lanczos, one k-batched H·X launch per step).  opts as for omen_eigs with block = 1
 * and which LOWEST or NEAREST; for NEAREST, tol bounds the H residual estimated from the
 * folded residual.  evals_host [nk][nev] ascending per k; evecs_dev [nk][nev][nrows] or NULL;
 * info aggregates over k (max residual and bound).  ENOCONV if some k did not converge. */
omen_status omen_eigs_kbatch(omen_ctx* ctx, const omen_ham* ham, int nk, const double* k_host,
                             const omen_eig_opts* opts, double* evals_host, void* evecs_dev,
                             omen_eig_info* info);

/* The same over several structures: every (structure, wave vector) pair is its own problem,
 * all in lockstep, one H·X launch per step for all of them.  opts.basis + 1 must not exceed
 * the smallest structure's rows.  evals_host [sum nk_i][nev] in item order, then k order;
 * evecs_dev (or NULL): per problem nev vectors of that structure's rows, problems one after
 * another in the same order. */
omen_status omen_eigs_kbatch_multi(omen_ctx* ctx, int nitems, const omen_kbatch_item* items,
                                   const omen_eig_opts* opts, double* evals_host, void* evecs_dev,
                                   omen_eig_info* info);

/* ---- charge, Poisson, self-consistency (paper Section III-A items 2-3) ------------------- */

typedef struct {
  int nx, ny;                /* grid points along the periodic x and y directions */
  int nz;                    /* intervals along z; unknowns at z_k = k*Lz/nz, k = 1..nz-1 */
  double Lx_nm, Ly_nm, Lz_nm;
  double eps_r;              /* relative permittivity (Si: 11.7) */
} omen_grid;
/* Grid arrays (rho, phi) hold the interior unknowns, index ((k-1)*ny + j)*nx + i.
 * phi = 0 V on the planes z = 0 and z = Lz. */

typedef struct {
  double rtol;               /* stop when ||r|| <= rtol ||b|| (b - A x in FP64 in both forms) */
  int max_iter;
  int precision;             /* OMEN_F64: FP64 iterations.  OMEN_F32_REFINE64: FP32 iterations
                                whose residual is replaced by the FP64 one b - A x after every
                                10x drop (reliable updates); x, the stopping test and the answer
                                stay FP64.  Zero-initialised options give OMEN_F64. */
} omen_cg_opts;

typedef struct {
  int iterations;
  int converged;
  double rel_residual;       /* ||r|| / ||b|| at exit */
  double seconds;
} omen_solve_info;

/* Solve -div(eps0 eps_r grad phi) = rho (7-point finite differences, periodic x and y,
 * phi = 0 at both z ends) by conjugate gradients, all iterations in one cooperative launch
 * (paper: finite-difference Poisson solver, Section III-A item 3), in FP64 or with FP32
 * iterations and FP64 residual replacement (opts->precision).
 * rho_dev: C/m^3; phi_dev: V, initial guess in, solution out (rho = 0 gives phi = 0).
 * ENOCONV at max_iter; EINVAL for a grid of 2^31 or more unknowns or another precision. */
omen_status omen_poisson(omen_ctx* ctx, const omen_grid* grid, const double* rho_dev, double* phi_dev,
                         const omen_cg_opts* opts, omen_solve_info* info);

/* The same solve for callers that must not allocate device memory (the paper has no
 * counterpart).  Some applications own all device memory through their own allocator, or
 * forbid any allocation once their run has started, so a library may not call cudaMalloc
 * behind their back.  This entry point allocates nothing: its CG work vectors live in one
 * statically sized device array that every GPU loading the library holds until the process
 * exits (OMEN_POISSON_STATIC_MAX_UNKNOWNS unknowns, about 6.4 MB).  The caller still passes
 * rho_dev and phi_dev (initial guess in, solution out) and the stream to work on; the
 * current device is used.
 *  - Every call looks up the array's device address on the current device (a pointer kept
 *    across a cudaDeviceReset would be stale); the first call on a device loads the library's
 *    device code there, so make that first call before any stream capture.
 *  - Grids with more than OMEN_POISSON_STATIC_MAX_UNKNOWNS interior unknowns
 *    (nx*ny*(nz-1)) are rejected with OMEN_EINVAL, and so is opts->precision other than
 *    OMEN_F64 (the iterations here are FP64); other argument errors also return
 *    OMEN_EINVAL, CUDA failures OMEN_ECUDA, hitting max_iter OMEN_ENOCONV.  No message
 *    is recorded (there is no context).
 *  - All calls share the one array, which keeps the last call's contents; every word is
 *    written before it is read, so nothing carries over.  Calls whose work overlaps on the
 *    GPU (other streams or threads) race on the array and must be serialised by the caller.
 *  - The call waits for its stream before returning (it reads the iteration count back). */
#define OMEN_POISSON_STATIC_MAX_UNKNOWNS 262144
omen_status omen_poisson_static(const omen_grid* grid, const double* rho_dev, double* phi_dev,
                                const omen_cg_opts* opts, omen_solve_info* info, void* cuda_stream);

/* Newton–Raphson nonlinear Poisson (paper Section III-A item 3: the converged potential of the
 * Poisson solver is obtained iteratively by Newton–Raphson).  The eigenstates computed in the
 * potential phi_in are frozen; the electrons respond to a change of potential by a local shift of
 * the levels (the predictor of Trellakis et al., J. Appl. Phys. 81, 7880 (1997)):
 *   n_i(phi) = sum_n W_ni f((E_n - u_i - E_F)/kT),  u_i = phi(r_i) - phi_in(r_i)
 * (potential at the atoms by trilinear interpolation, as omen_gather), and
 *   -div(eps0 eps_r grad phi) = rho_D - q * deposit(n(phi))
 * (cloud-in-cell deposit as omen_deposit) is solved by Newton–Raphson with the exact Jacobian,
 * each step a conjugate-gradient solve in one cooperative launch. */
typedef struct {
  int nstates;
  const double* E_host;      /* [nstates] levels (eV) in the potential phi_in */
  const double* W_dev;       /* [nstates][natoms] electrons each state puts on each atom when full
                                (spin and k weight included; 0 for states that hold none), e.g.
                                from omen_state_weights */
  double E_F;                /* eV */
  double kT;                 /* eV, > 0 */
  const double* phi_in_dev;  /* grid potential the states were computed in (V) */
} omen_frozen_states;

typedef struct {
  double tol_V;              /* stop when the largest change of a Newton step is below tol_V */
  int max_iter;              /* Newton steps */
  omen_cg_opts cg;           /* each step's CG on the Jacobian (relative residual, iterations;
                                the precision field is not used: these iterations are FP64) */
} omen_newton_opts;

typedef struct {
  int iterations;            /* Newton steps taken */
  int converged;
  double last_step_V;        /* max |change| of the last step */
  long long cg_iterations;   /* CG iterations over all steps */
  double seconds;
} omen_newton_info;

/* Solve the nonlinear Poisson equation above on grid for the structure lat.  rho_d_dev: fixed
 * (donor) charge density on the interior unknowns (C/m^3); phi_dev: start in (e.g. phi_in),
 * root out.  Allocates its work (maps and vectors, about 24 words per atom and 5 per unknown)
 * on ctx's stream; synchronous.  EINVAL for bad arguments, ENOCONV when a CG solve or the
 * Newton iteration hits its limit (phi_dev holds the last iterate), ENUMERIC on a non-finite
 * step. */
omen_status omen_poisson_newton(omen_ctx* ctx, const omen_lattice* lat, const omen_grid* grid,
                                const omen_frozen_states* states, const double* rho_d_dev, double* phi_dev,
                                const omen_newton_opts* opts, omen_newton_info* info);

/* W_dev[n][i] = weight_host[n] * sum_o |psi_n(o*natoms + i)|^2 for nstates FP64 (double or
 * complex128) vectors psi_dev [nstates][nrows] of a tight-binding Hamiltonian: the W of
 * omen_frozen_states (weight = spin degeneracy times k weight, 0 for states that hold no
 * electrons).  EUNSUPPORTED for an effective-mass Hamiltonian. */
omen_status omen_state_weights(omen_ctx* ctx, const omen_ham* ham, const void* psi_dev, int nstates,
                               const double* weight_host, double* W_dev);

/* n_atom_dev[i] += weight * sum_n occ_host[n] * sum_o |psi_n(o*natoms + i)|^2 for nstates FP64
 * (double or complex128) vectors psi_dev [nstates][nrows] of ham (paper: charge from the
 * filled states, Section III-A item 2).  The squares are summed in double-float arithmetic
 * (about 1e-14 relative) on the FP32 pipe: amplitude components below 2^-83 in magnitude
 * count as zero, components of 2^32 or more overflow, and non-finite ones give NaN. */
omen_status omen_density_accum(omen_ctx* ctx, const omen_ham* ham, const void* psi_dev, int nstates,
                               const double* occ_host, double weight, double* n_atom_dev);

/* Cloud-in-cell (trilinear) deposit of per-atom charge q_atom_dev (C) onto the grid nodes,
 * divided by the cell volume: rho_dev (C/m^3) is overwritten.  Charge landing on the z = 0 or
 * z = Lz planes is dropped (grounded).  Atom positions come from the structure. */
omen_status omen_deposit(omen_ctx* ctx, const omen_lattice* lat, const omen_grid* grid,
                         const double* q_atom_dev, double* rho_dev);
/* Trilinear interpolation of phi (boundary planes at 0 V) to every atom: phi_atom_dev [natoms]. */
omen_status omen_gather(omen_ctx* ctx, const omen_lattice* lat, const omen_grid* grid,
                        const double* phi_dev, double* phi_atom_dev);

/* Fermi level by bisection: sum_i g_i f((E_i - E_F)/kT) = n_target with g_i = level_weight[i]
 * (k weight times spin degeneracy).  Host only; no device use.  EINVAL if n_target is not
 * reachable with the given levels. */
omen_status omen_fermi_level(const double* E, const double* level_weight, int n, double n_target,
                             double kT, double* E_F);

typedef struct {
  const omen_lattice* lat;
  const omen_tb_params* params;
  int precision;             /* eigen-solve precision (OMEN_F64 or OMEN_F32_REFINE64) */
  const omen_grid* grid;
  const double* donor_rho_dev; /* fixed positive charge density on the grid (C/m^3) */
  double n_electrons;        /* electrons per supercell (charge neutrality) */
  double kT;                 /* eV */
  int nk;                    /* k points (supercell Bloch vectors, 1/nm) and weights (sum 1) */
  const double* k_host;      /* [nk][3] */
  const double* kw_host;     /* [nk] */
  int nev;                   /* states per k nearest sigma (folded spectrum) */
  double sigma;              /* eV */
  double e_cut;              /* only states above e_cut hold electrons (conduction band) */
  double eig_tol;
  int eig_block, eig_basis, eig_max_iter;
  double mix;                /* mixing weight beta */
  int mix_history;           /* 0: linear mixing phi <- phi + beta F, F = phi_out - phi;
                                m > 0: Anderson mixing over the last m iterations */
  double tol_V;              /* stop when max |phi_out - phi| < tol_V */
  int max_iter;
  omen_cg_opts cg;
  int poisson_newton;        /* 0: phi_out solves the linear Poisson equation with the states'
                                charge; 1: phi_out is the root of the nonlinear Poisson equation
                                with the frozen states' predicted charge (omen_poisson_newton,
                                steps to min(1e-9, tol_V/100) V, CG options as above) */
} omen_scf_desc;

typedef struct {
  int iterations;
  int converged;
  double dV_inf;             /* last max |phi_out - phi| (V) */
  double E_F;                /* eV */
  long long hx_count;        /* H·X products over all eigen-solves */
  double seconds;
  double eig_seconds, poisson_seconds;
} omen_scf_info;

/* Self-consistent Schrödinger–Poisson loop (paper Section III-A): potential -> onsite
 * U = -phi at the atoms -> eigenstates per k -> Fermi level by neutrality -> electron charge
 * -> Poisson (linear, or Newton–Raphson with the frozen-state predictor) -> mixing (linear or
 * Anderson), until max |phi_out - phi| < tol_V.  phi_dev: grid potential, start
 * value in (zeros = zero-field start), converged potential out.  ENOCONV at max_iter;
 * ENUMERIC if the highest computed state of some k is occupied above 1e-12 (nev too small). */
omen_status omen_scf(omen_ctx* ctx, const omen_scf_desc* desc, double* phi_dev, omen_scf_info* info);

/* ---- learned warm start (no counterpart in the paper) ------------------------------------ */
/* A 3-layer perceptron maps the doping profile to the self-consistent potential, giving the
 * Schrödinger–Poisson loop (Section III-A) a start closer to its fixed point than zero field.
 * x (n_in) -> tanh(W1 x + b1) -> tanh(W2 . + b2) -> W3 . + b3 (n_out).  BF16 weight copies are
 * used in every product with FP32 accumulation; FP32 master weights take Adam updates.
 * Parameters on the host: W1 [n_hidden1][n_in], b1, W2 [n_hidden2][n_hidden1], b2,
 * W3 [n_out][n_hidden2], b3, concatenated, FP32. */
typedef struct omen_mlp omen_mlp;
typedef struct {
  int n_in, n_hidden1, n_hidden2, n_out;   /* 256, 512, 512, 256 */
  double feat_log10_shift;   /* feature x_j = (log10(max(N_D(z_j), 1e15 m^-3)) - shift) / scale */
  double feat_log10_scale;
  double target_scale;       /* output y_j = phi(z_j) [V] / target_scale */
} omen_mlp_desc;
/* Profiles are sampled at z_j = (j + 1/2) Lz / n from the lateral mean of the grid planes
 * (linear interpolation, 0 on the grounded planes). */

omen_status omen_mlp_create(omen_ctx* ctx, const omen_mlp_desc* desc, const float* params_host, omen_mlp** out);
void omen_mlp_free(omen_mlp* mlp);
long long omen_mlp_param_count(const omen_mlp* mlp);
/* FP32 master parameters, or (bf16_rounded = 1) the weights as the products use them. */
omen_status omen_mlp_get_params(omen_ctx* ctx, const omen_mlp* mlp, float* params_host, int bf16_rounded);
/* Y_dev [batch][n_out] = network(X_dev [batch][n_in]). */
omen_status omen_mlp_forward(omen_ctx* ctx, omen_mlp* mlp, const float* X_dev, int batch, float* Y_dev);
/* Gradients of the mean squared error w.r.t. every parameter (host, parameter layout) and the
 * loss, without updating. */
omen_status omen_mlp_gradients(omen_ctx* ctx, omen_mlp* mlp, const float* X_dev, const float* T_dev, int batch,
                               float* grad_host, float* loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error. */
omen_status omen_mlp_train_step(omen_ctx* ctx, omen_mlp* mlp, const float* X_dev, const float* T_dev, int batch,
                                double lr, float* loss_host);
/* Features of a donor density on the grid (C/m^3) -> x_dev [n_in]; targets of a potential on
 * the grid (V) -> t_dev [n_out]. */
omen_status omen_mlp_features(omen_ctx* ctx, const omen_mlp* mlp, const omen_grid* grid, const double* donor_rho_dev,
                              float* x_dev);
omen_status omen_mlp_targets(omen_ctx* ctx, const omen_mlp* mlp, const omen_grid* grid, const double* phi_dev,
                             float* t_dev);
/* Start potential for omen_scf: network(features(donor_rho)) interpolated onto the grid planes
 * (0 V on the grounded planes), the same on every lateral point: phi_dev [(nz-1)*ny*nx]. */
omen_status omen_mlp_warm_start(omen_ctx* ctx, omen_mlp* mlp, const omen_grid* grid, const double* donor_rho_dev,
                                double* phi_dev);

/* omen_scf from the network's start (omen_mlp_warm_start on d->donor_rho_dev), with the
 * zero-field start as the fallback: if that loop returns ENOCONV or ENUMERIC, phi_dev is reset to
 * zero and omen_scf runs again.  *fallback (may be NULL) = 1 when the result comes from the
 * zero-field run; info then counts both runs' time and products, and its iterations those of the
 * zero-field run.  d->donor_rho_dev is required. */
omen_status omen_scf_learned(omen_ctx* ctx, const omen_scf_desc* d, omen_mlp* mlp, double* phi_dev,
                             omen_scf_info* info, int* fallback);

#ifdef __cplusplus
}
#endif
#endif /* OMEN_H */
