/*
 * gint.h -- C ABI of libgint: uniform-grid integration of numerical atomic
 * orbitals (NAOs) at the Gamma point on one GB300 GPU (sm_103a).
 *
 * The operations are those of the paper's Sec. 3.3.1 ("Uniform Grid Integration
 * for Usual Quantities"): with periodised orbitals
 *     Phi_mu(r) = sum_R phi_mu(r - tau_I - R),   phi_mu = f_{I l zeta}(|r|) Y_lm(r^)   (Eqs. 1-2, k = 0)
 * on the grid r_g = (i/n1) a1 + (j/n2) a2 + (k/n3) a3 with weight w = |det A| / (n1 n2 n3):
 *     density         rho_g    = sum_{mu nu} D_{mu nu} Phi_mu(r_g) Phi_nu(r_g)
 *     local H         H_{mu nu} = sum_g w V_g Phi_mu(r_g) Phi_nu(r_g)
 *     local Pulay     F_I      = - dE/dtau_I,  E = sum_g w V_g rho_g  (V fixed)
 *
 * Conventions
 *   - Units: Bohr, Hartree.  Cell rows are the lattice vectors a1, a2, a3.
 *   - Grid arrays (rho, V) are float64, C order [n1][n2][n3] (k fastest), device memory.
 *   - Orbitals of an atom follow its species' radial list in the given order; each radial
 *     with angular momentum l contributes 2l+1 orbitals, m ordered 0, +1, -1, +2, -2
 *     (real, orthonormal Y_lm without the Condon-Shortley sign; l <= 2).
 *   - Radial tables hold R(r_k) (including the r^l factor) and R'(r_k) at r_k = k dr; the
 *     library interpolates with cubic Hermite polynomials; R = 0 for r >= rc.
 *   - Matrices (D in, H out) are stored as atom-pair blocks.  Pair p = (I, J) exists when
 *     some lattice image of J lies closer to I than rcut(I) + rcut(J) + skin; both (I, J) and
 *     (J, I) are stored.  Block p is row-major norb(I) x norb(J) at element offset
 *     pair_off[p] of a float64 device array of nblock_elems elements.  Pairs are sorted by
 *     I, then J.  D must be symmetric (block (J, I) = block (I, J)^T).
 *
 * Ownership and streams
 *   - gint_create copies everything it needs; the caller's host arrays may be freed after.
 *   - The handle owns its device state (tables, neighbour lists, workspace).  Compute calls
 *     take caller-owned device pointers (non-owning) and allocate nothing.
 *   - Compute calls are asynchronous on the given CUDA stream (NULL: legacy default stream).
 *     Calls on one handle must not overlap (they share the handle's workspace).
 *
 * Errors: every function returns GINT_OK (0) or a negative GINT_E* code; no exceptions
 * cross the ABI.  gint_strerror() names a code.
 */
#ifndef GINT_H
#define GINT_H

#ifdef __cplusplus
extern "C" {
#endif

#define GINT_OK 0
#define GINT_EINVAL (-1)     /* bad argument or descriptor */
#define GINT_ENOMEM (-2)     /* device allocation failed */
#define GINT_ECUDA (-3)      /* a CUDA runtime call failed */
#define GINT_ETIMEDOUT (-4)  /* a bounded device wait gave up */
#define GINT_EDEVICE (-5)    /* a kernel reported an inconsistency through the device error word */
#define GINT_ECAPACITY (-6)  /* a brick holds more orbitals/atoms than the kernels support */
#define GINT_ESKIN (-7)      /* atoms moved so that a pair outside the block set now overlaps */
#define GINT_EUNSUPPORTED (-8) /* precision mode or feature not available on this device */
#define GINT_EBUSY (-9)      /* the serving queue is full or the task's handle has a job in flight */

/* Precision of the brick contractions.  The charge and energy reductions and the per-atom force
 * reduction are float64 in every mode.  The cross-brick reduction of H is float64 in the FP64 mode;
 * with the tensor-core modes the per-brick float32 tiles are summed as double-float pairs (error-free
 * two-sum into a float32 hi + lo pair, relative error about n^2 2^-48 for n bricks) and the pair is
 * combined in float64.
 * GINT_F16X3 forces (gint_force, and force tasks of gint_run_batch) split orbitals and D in fixed point
 * instead: hi = the nearest integer at a common scale (so the tensor core's float32 accumulation of
 * hi * hi is exact), lo = the float16 remainder, and four products hi*hi + hi*lo + lo*hi + lo*lo. */
#define GINT_FP64 0  /* float64 everywhere (CUDA cores) */
#define GINT_FP32 1  /* float32 orbitals and CUDA-core contractions */
#define GINT_F16X3 2 /* float32 orbitals; tensor-core contractions on operands split into two float16
                        parts (hi + lo, 22 significant bits, power-of-two scaled), products
                        hi*hi + hi*lo + lo*hi, float32 accumulation */
#define GINT_F16X1 3 /* as GINT_F16X3 with the hi*hi product only (about 3 significant digits) */

typedef struct gint_radial {
  int l;            /* angular momentum, 0..2 */
  int npts;         /* number of knots (>= 2) */
  double dr;        /* knot spacing (> 0) */
  double rc;        /* support radius: R = 0 for r >= rc; rc <= (npts-1) dr */
  const double *f;  /* host [npts]: R(k dr) including r^l */
  const double *df; /* host [npts]: R'(k dr) */
} gint_radial;

typedef struct gint_species {
  int nradial;               /* number of radial functions (1..16) */
  const gint_radial *radial; /* host [nradial] */
} gint_species;

typedef struct gint_desc {
  double cell[9];          /* row-major a1, a2, a3 (Bohr) */
  int natoms;              /* >= 1 */
  const double *pos;       /* host [natoms][3] Cartesian (Bohr) */
  const int *species;      /* host [natoms], 0..nspecies-1 */
  int nspecies;            /* 1..8 */
  const gint_species *sp;  /* host [nspecies] */
  int n1, n2, n3;          /* grid (each >= 1) */
  double skin;             /* extra pair-set margin (Bohr, >= 0) for later gint_set_positions */
} gint_desc;

typedef struct gint_handle gint_handle;

/* Builds the handle on the current CUDA device: radial tables, the grid-brick -> atom
 * neighbour lists (device kernels), the atom-pair block set and the workspace (the
 * paper's GintInfo / MeshGrid / BigGrid set-up, Sec. 3.3.1 and Fig. 2).  Synchronous.
 * Returns GINT_EINVAL for a malformed descriptor, GINT_ENOMEM / GINT_ECUDA on CUDA failure,
 * GINT_ECAPACITY if a brick exceeds the kernels' limits.  *out is NULL on failure. */
int gint_create(const gint_desc *desc, gint_handle **out);

/* Frees the handle and all its device memory.  NULL is accepted. */
int gint_destroy(gint_handle *h);

/* Sizes of the block layout: total orbitals, number of pairs, float64 elements of a
 * block array (the sparse atom-pair blocks of D and H of paper Sec. 3.3.1, R summed at the Gamma
 * point).  Any output pointer may be NULL. */
int gint_layout(const gint_handle *h, int *norb, int *npairs, long long *nblock_elems);

/* Copies the pair list to host arrays: pair_IJ [npairs][2], pair_off [npairs + 1]. */
int gint_pairs(const gint_handle *h, int *pair_IJ, long long *pair_off);

/* Work statistics of the current geometry (host outputs, any may be NULL):
 *   W         = sum_g n_g^2, n_g = orbitals whose support covers grid point g (exact,
 *               ordered pairs; the algorithmic work of one rho or H pass);
 *   W_exec    = sum over bricks of 128 * norb(brick)^2 (the padded work a brick kernel sees);
 *   nbricks, max orbitals of a brick, max atoms of a brick. */
int gint_stats(const gint_handle *h, double *W, double *W_exec, long long *nbricks, int *max_brick_orb,
               int *max_brick_atoms);

/* Diagnostic: the grid-brick -> atom neighbour lists of the current geometry (the paper's BigGrid
 * neighbour relation, Sec. 3.3.1 and Fig. 2), copied to host arrays.  Brick b = (bi nb2 + bj) nb3 + bk
 * (nb_i = ceil(n_i / brick_i), bricks of 4 x 4 x 8 points) covers grid points [4 bi, 4 bi + 4) x
 * [4 bj, 4 bj + 4) x [8 bk, 8 bk + 8) (clipped to the grid).  An entry is a lattice image tau_I + R of an
 * atom whose support sphere (|r - tau_I - R| < rcut(I)) strictly contains at least one grid point of
 * the brick; the entries of one atom form a slot, the slots of a brick are sorted by atom.  Outputs
 * (host, any may be NULL; pass NULL arrays first to learn the counts):
 *   nslots, nentries;  b_off [nbricks + 1]: slots of brick b are [b_off[b], b_off[b + 1]);
 *   slot_atom [nslots];  slot_ent [nslots + 1]: entries of slot s are [slot_ent[s], slot_ent[s + 1]);
 *   ent_pos [nentries][3]: Cartesian tau_I + R of each entry.
 * Synchronous.  GINT_ECUDA if a copy fails. */
int gint_brick_lists(const gint_handle *h, long long *nslots, long long *nentries, long long *b_off, int *slot_atom,
                     long long *slot_ent, double *ent_pos);

/* Diagnostic: the periodised orbitals Phi_mu (Eqs. 1-2 at k = 0, all lattice images within the support)
 * and their gradients at arbitrary points, evaluated by the brick kernels' own evaluators:
 * GINT_FP64 (the float64 CUDA-core evaluator) or GINT_F16X3 (the tensor-core path's float32 evaluator:
 * double-float distance and knot parameter, float32 Hermite interpolation with derivative differences
 * formed in float64, float32 Y_lm).  pts [npts][3] (host, Cartesian Bohr); phi [npts][norb] and grad
 * [npts][norb][3] (host outputs, grad may be NULL).  Synchronous; allocates temporary device memory.
 * GINT_EUNSUPPORTED for other precisions. */
int gint_orbitals(gint_handle *h, int precision, long long npts, const double *pts, double *phi, double *grad);

/* Device memory held by the handle (tables, neighbour lists, workspace), in bytes (host
 * output).  The footprint that a serving loop counts against its HBM budget. */
int gint_memory(const gint_handle *h, long long *device_bytes);

/* Replaces the atom positions from a DEVICE array [natoms][3] and rebuilds the neighbour
 * lists on the device (the BigGrid neighbour relation of paper Sec. 3.3.1 and Fig. 2, renewed as
 * the ions move in the Ehrenfest dynamics of Sec. 2).  The pair set stays fixed: GINT_ESKIN if a
 * pair outside it now overlaps.  When every brick keeps its atoms, only the tensor-core path's
 * per-brick plan records are rebuilt; otherwise its layouts are rebuilt as at creation.  Results
 * equal those of a handle created at the new positions.  Synchronises the stream. */
int gint_set_positions(gint_handle *h, const double *pos_dev, void *stream);

/* Density pass: rho [n1 n2 n3] (device, overwritten) from D blocks (device). */
int gint_rho(gint_handle *h, int precision, const double *D_blocks, double *rho, void *stream);

/* Local-Hamiltonian pass: H blocks (device, overwritten) from V [n1 n2 n3] (device). */
int gint_vlocal(gint_handle *h, int precision, const double *V, double *H_blocks, void *stream);

/* Cross-brick reduction of the tensor-core local-H pass (GINT_F16X3 / GINT_F16X1; the FP64 and FP32
 * paths are unaffected).  The per-brick tiles are float32 (the tensor cores' accumulators); they are
 * summed over the bricks in a fixed order
 *   GINT_REDUCE_DOUBLE_FLOAT (default): as double-float pairs (error-free float32 additions into a
 *     hi + lo pair), the pairs combined in float64: summation error about n^2 2^-48 relative for n
 *     bricks, far below the float32 rounding of the tiles;
 *   GINT_REDUCE_FP64: every tile value converted to float64 and added in float64 (the float64 pipe
 *     of the GB300 makes this the slower reduction).
 * Both are deterministic.  Applies to later gint_vlocal / gint_vlocal_R / gint_run_batch calls on h
 * (and to the server's jobs that use h).  GINT_EINVAL for another mode. */
#define GINT_REDUCE_DOUBLE_FLOAT 0
#define GINT_REDUCE_FP64 1
int gint_set_reduction(gint_handle *h, int mode);

/* Local H per lattice vector (paper Sec. 2, H_{mu nu}(R); Sec. 3.3.1, the local-potential matrix
 * element between phi_mu at tau_I and phi_nu at tau_J + R): keys (I, J, R) with
 * R = n1 a1 + n2 a2 + n3 a3, one norb(I) x norb(J) row-major block per key, keys sorted by
 * (I, J, n1, n2, n3); for each key (I, J, R) the key (J, I, -R) exists and H_JI(-R) = H_IJ(R)^T.
 * Summed over R, the blocks of (I, J) give the Gamma-point block of gint_vlocal.
 *
 * gint_layout_R: host outputs (any may be NULL): the number of keys, the float64 elements of an
 * H(R) array, and pointers to library-owned host arrays keys [nkeys][5] (I, J, n1, n2, n3) and
 * key_off [nkeys + 1] (element offset of each block), valid until the positions change or the
 * handle is destroyed.  The tables are built on the first call (synchronous).
 * Where some brick sees two lattice images of one atom (a cell shorter than about twice the orbital
 * cutoff plus a brick), the handle's brick tiles mix several R; there the first call also builds an
 * unfolded twin of the handle (same descriptor and pair layout, one brick slot per atom image;
 * counted by gint_memory, moved by gint_set_positions), and the per-R calls run on it.
 * GINT_ECAPACITY if the twin's bricks exceed the local-H kernel's limit of 288 padded orbital columns
 * (18 images of 13-orbital atoms per brick; the 8-atom cubic Si cell needs 16). */
int gint_layout_R(gint_handle *h, int *nkeys, long long *nblock_elems, const int **keys, const long long **key_off);

/* Local-Hamiltonian pass per lattice vector: H_R [nblock_elems of gint_layout_R] (device,
 * overwritten) from V [n1 n2 n3] (device).  Tensor-core precisions only (GINT_F16X3, GINT_F16X1;
 * others: GINT_EUNSUPPORTED): the same brick pass as gint_vlocal, reduced per (I, J, R). */
int gint_vlocal_R(gint_handle *h, int precision, const double *V, double *H_R, void *stream);

/* Bloch sums (paper Sec. 2): H(k) = sum_R e^{i k.R} H(R) for nk k points, each in the Gamma-point
 * block layout of gint_vlocal, complex float64 interleaved (re, im): H_k [nk][2 nblock] (device,
 * overwritten), from H_R (device, as written by gint_vlocal_R).  kfrac [nk][3] (host) is each k in
 * reciprocal-lattice units (k = kf1 b1 + kf2 b2 + kf3 b3, a_i . b_j = 2 pi delta_ij), so
 * k.R = 2 pi (kf . n).  Up to 8 k points share one pass over H(R).  At kfrac = 0 it is the Gamma
 * block. */
int gint_bloch(gint_handle *h, const double *H_R, int nk, const double *kfrac, double *H_k, void *stream);

/* Velocity-gauge nonlocal projector overlaps (paper Sec. 3.3.2, "Spherical Grid Integration for
 * Nonlocal Potentials"): P_{j mu}^{IJ}(A) = <beta_{I j}| e^{-i A.r} |Phi_{J mu}>, the integral of
 * beta_{I j}(r - tau_I) e^{-i A.r} Phi_{J mu}(r) on a grid centred on tau_I (140 Gauss-Legendre radial
 * nodes on [0, rc_beta] and a degree-17 angular rule: 9 Gauss-Legendre nodes in cos(theta) x 18
 * azimuths, standing in for the paper's 110-point Lebedev-Laikov rule).  Phi is the orbital summed over
 * the lattice images of J (Gamma point); r is the Cartesian position (the phase is not periodic).
 *
 * gint_set_projectors: projector radial tables per species (host, same species order as the
 * descriptor; a species may have none), f including r^l, l <= 2, beta_j = f(r) Y_lm in the orbitals'
 * convention.  Builds the pair list (I, J) of atoms whose orbitals reach I's projectors.  Synchronous.
 * GINT_EUNSUPPORTED if an orbital species has more than 16 orbitals.
 * gint_psibeta_layout: host outputs (any may be NULL): number of pairs, complex elements, and pointers
 * to library-owned host arrays pairs [npairs][2] (I, J) and off [npairs + 1]; pair p's block is
 * nbeta(I) x norb(J) row-major at off[p] (projector functions in the order of the radials, m as for
 * orbitals).  GINT_EINVAL before gint_set_projectors.
 * gint_psibeta: A [3] (host, atomic units), out [2 nelems] (device, overwritten, re / im interleaved),
 * float64 throughout. */
int gint_set_projectors(gint_handle *h, int nspecies, const gint_species *proj);
int gint_psibeta_layout(const gint_handle *h, int *npairs, long long *nelems, const int **pairs,
                        const long long **off);
int gint_psibeta(gint_handle *h, const double *A, double *out, void *stream);

/* Dense steps of real-time propagation around the grid passes (paper Sec. 2): the density matrix
 * from coefficients and occupations, and one Crank-Nicolson step of the coefficients, in float64 on
 * the library's own kernels (a tiled GEMM, a blocked L D L^T factorisation without pivoting and its
 * triangular solves).  A context holds all
 * buffers for an n x n problem with nocc states (allocated by gint_cn_create on the current device),
 * so the compute calls allocate nothing.  Matrices are float64 n x n, symmetric (any order); psi is
 * complex float64 n x nocc column-major (state j is psi[j n .. j n + n)), re / im interleaved; all
 * device pointers, caller-owned; the calls are asynchronous on `stream` and must not run
 * concurrently on one context.
 *
 * gint_cn_step: psi_out = (S + i dt/2 H)^{-1} (S - i dt/2 H) psi (psi_out must not alias psi),
 * computed as 2 X - psi with (S + i dt/2 H) X = S psi; S + i dt/2 H (complex symmetric, positive
 * definite Hermitian part S) is factored as L D L^T without pivoting.
 * gint_dm_build: D = Re(psi diag(f) psi^dagger), f [nocc] (device) occupations; D is symmetric bit
 * for bit.
 * gint_dm_build_f16x3: the same D on the tensor cores: D = A B^T with A_ik = f_s psi_is, B_ik = psi_is
 * (k = 2 s + real / imaginary part), each operand scaled by a power of two and split into float16
 * hi + lo, three float16 products per term (lo lo dropped).  The hi hi products of each chunk of 64 k
 * go to a fresh float32 tensor-memory accumulator, which is added into float32 Kahan sums; the
 * cross products share one accumulator; the parts are combined in float64.  D is symmetric bit for
 * bit; its error stays within about 3 * 2^-22 of max_i sum_s |f_s| |psi_is|^2 (measured up to
 * 2.8e-7).  Occupations of any sign; psi 16-byte aligned (as for every complex128 array here); no
 * allocation.
 * gint_cn_info: the LAPACK-style info of the last factorisation (0: success; i > 0: the pivot d_i of
 * L D L^T is zero or not finite, or for gint_edm not positive);
 * synchronous; returns GINT_ETIMEDOUT (once) when a bounded wait of the tensor-core build gave up.  The
 * D of that call is then undefined; and since a CTA whose final completion wait also gave up releases
 * its tensor memory with MMAs possibly still in flight, destroy the context after GINT_ETIMEDOUT rather
 * than reuse it. */
typedef struct gint_cn gint_cn;
int gint_cn_create(int n, int nocc, gint_cn **out);
int gint_cn_destroy(gint_cn *c);
int gint_cn_step(gint_cn *c, const double *S, const double *H, double dt, const double *psi, double *psi_out,
                 void *stream);
int gint_dm_build(gint_cn *c, const double *psi, const double *f, double *D, void *stream);
int gint_dm_build_f16x3(gint_cn *c, const double *psi, const double *f, double *D, void *stream);
int gint_cn_info(gint_cn *c, int *info);

/* Energy-density matrix E = (S^{-1} H D + D H S^{-1}) / 2 (the overlap part of the forces needs it):
 * S (positive definite), H, D real symmetric n x n (device), E (device, overwritten); X = H D, then
 * S X' = X by L D L^T of S, E = (X' + X'^T) / 2 (bit-for-bit symmetric), with the context's buffers
 * (gint_cn_info reports a non-positive pivot as i > 0). */
int gint_edm(gint_cn *c, const double *S, const double *H, const double *D, double *E, void *stream);

/* Local Pulay forces F [natoms][3] (device, overwritten) = -dE/dtau for E = sum_g w V rho.
 * If rho is not NULL the density is written as well (same pass). */
int gint_force(gint_handle *h, int precision, const double *D_blocks, const double *V, double *F, double *rho,
               void *stream);

/* One unit of work for gint_run_batch: the passes of one system (its own handle).  Outputs
 * that are NULL are not computed:
 *   rho      [n1 n2 n3]  density (needs D_blocks)
 *   H_blocks [nblock]    local H (needs V)
 *   F        [natoms][3] local Pulay forces (needs D_blocks and V); rho is written in the same
 *                        pass if it is not NULL
 * All pointers are caller-owned device memory; the handle's workspace is used, so one handle may
 * appear only once per batch and must not be used concurrently elsewhere. */
typedef struct gint_task {
  gint_handle *h;
  const double *D_blocks;
  const double *V;
  double *rho;
  double *H_blocks;
  double *F;
} gint_task;

/* Runs the tasks of several systems together (the batched dense-tile reformulation of paper
 * Sec. 3.3.1, here across systems as well as bricks; a serving loop's batches).  With the
 * tensor-core precisions the bricks of all tasks (density / force bricks and local-H bricks) are
 * items of ONE persistent launch, up to 32 tasks per launch (more are split into groups of 32);
 * the per-pair H reduction and the per-call preparation are one launch each for the group.
 * Results equal those of the single-system calls on each handle, because every brick is computed
 * the same way whatever else shares the launch.  The FP64 / FP32 precisions run the tasks one
 * after another (separate launches).  Asynchronous on `stream`.  Every handle must live on the
 * same device and have been created with the same species list (identical radial metadata);
 * otherwise GINT_EINVAL, as for a repeated handle or a missing input. */
int gint_run_batch(const gint_task *tasks, int ntasks, int precision, void *stream);

/* gint_run_batch that also records two caller-created CUDA events (cudaEvent_t, may be NULL) on
 * `stream`: ev_start right before the first brick-kernel launch and ev_stop right after the
 * last (FP64 / FP32: around all of the batch's kernels), so that the brick kernels can be timed
 * without the per-call preparation and reduction launches. */
int gint_run_batch_timed(const gint_task *tasks, int ntasks, int precision, void *stream, void *ev_start,
                         void *ev_stop);

/* Continuous-batching server: ONE resident launch of the brick kernels drains a device work queue to
 * which jobs are appended while it runs, so a request that arrives while others are on the GPU starts
 * as soon as it is published, in the same residency, and its work overlaps theirs on the device.  A
 * job is one task (rho, H and, with forces, F of one system, as for gint_run_batch); its per-call
 * preparation (maxima and scales), D tiles, bricks and H reduction are all items of the resident
 * kernel, each waiting (bounded) for the items of its job that it depends on.  The kernel leaves after
 * idle_s seconds without work (or on gint_server_stop); submit and test relaunch it when needed.
 *
 * gint_server_create: precision GINT_F16X3 or GINT_F16X1; forces != 0 runs the force variant of the
 *   brick items (jobs may then ask for F; tasks without F get rho from the same pass).  Allocates its
 *   queue and host-mapped completion words on the current device.
 * gint_server_submit: publishes one task.  Its device inputs (D, V) must be complete in stream order
 *   on `stream` (the job starts after that stream's work submitted so far); outputs are written
 *   asynchronously.  Every task's handle must be on the server's device with the same species list.
 *   At most 64 jobs in flight and one job per handle at a time: GINT_EBUSY otherwise (test the
 *   earlier jobs and submit again).  *ticket identifies the job.  Does not block.
 * gint_server_test: *done = 1 once the job's results are in device memory (then read them on any
 *   stream); relaunches the resident kernel if it left with work outstanding; GINT_ETIMEDOUT /
 *   GINT_EDEVICE if an item's bounded wait gave up (the server cannot be used any more).
 * gint_server_stats: kernel launches so far and jobs submitted.
 * gint_server_stop: makes the resident kernel leave once idle and waits for it.
 * gint_server_destroy: stop, then free.
 * The paper has no serving layer; this is the serving pattern around its grid passes. */
typedef struct gint_server gint_server;
int gint_server_create(int precision, int forces, double idle_s, gint_server **out);
int gint_server_submit(gint_server *s, const gint_task *task, void *stream, long long *ticket);
int gint_server_test(gint_server *s, long long ticket, int *done);
int gint_server_stats(const gint_server *s, long long *launches, long long *jobs);
int gint_server_stop(gint_server *s);
int gint_server_destroy(gint_server *s);

/* Float64 reductions on the device, written to out_dev[0] (device):
 *   V != NULL: w * sum_g V_g rho_g  (the energy E whose derivative is the local Pulay force of
 *   paper Sec. 3.3.1);   V == NULL: w * sum_g rho_g (N_e = Tr(DS)). */
int gint_grid_dot(gint_handle *h, const double *V, const double *rho, double *out_dev, void *stream);

/* Float64 block-array dot product sum_p sum_e A[e] B[e] written to out_dev[0] (e.g. Tr(DH)). */
int gint_block_dot(gint_handle *h, const double *A_blocks, const double *B_blocks, double *out_dev, void *stream);

/* Waits for the stream and reports errors that kernels recorded in the handle's device error
 * word since the last check (GINT_ETIMEDOUT for a bounded wait that gave up, GINT_ECAPACITY,
 * GINT_EDEVICE); clears the word.  Compute calls are asynchronous, so such errors surface here. */
int gint_sync(gint_handle *h, void *stream);

/* Diagnostic: runs one tcgen05 kind::f16 MMA (M=128, N=n, K=16) per operand layout used by the
 * brick kernels on exactly representable integer data and returns the largest absolute deviation
 * from the exact product in *max_err (host).  n in {16, ..., 256}, multiple of 16.  Synchronous. */
int gint_tc_selftest(int n, double *max_err);

/* Float64 dot product that allocates no device memory (the paper has no counterpart; this
 * entry point exists for callers that cannot let a library allocate: applications whose device
 * memory is owned by their own pool allocator, or latency-critical loops that cannot accept the
 * implicit synchronisation of cudaMalloc / cudaFree).
 *   out_dev[0] = scale * sum_i a[i] * b[i]   (b == NULL: scale * sum_i a[i])
 * a, b, out_dev are caller-owned device pointers; the call is asynchronous on `stream`.  The sum
 * runs over fixed chunks of GINT_NOALLOC_CHUNK elements, so the result does not depend on the GPU.
 * Scratch: one float64 partial per chunk in a file-scope __device__ array of
 * GINT_NOALLOC_MAX_CHUNKS entries (32 KiB) that every GPU loading the library keeps until exit;
 * n above GINT_NOALLOC_MAX_CHUNKS * GINT_NOALLOC_CHUNK returns GINT_ECAPACITY.  The first call on
 * a device looks up the array's device address on that device (once per device, with it
 * current), so that first call should come before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (other streams, other host threads) race.
 * Returns GINT_EINVAL for a NULL a / out_dev or negative n, GINT_ECUDA on CUDA failure. */
#define GINT_NOALLOC_CHUNK 65536LL
#define GINT_NOALLOC_MAX_CHUNKS 4096
int gint_grid_dot_noalloc(const double *a, const double *b, long long n, double scale, double *out_dev,
                          void *stream);

/* Grid weight w = |det A| / (n1 n2 n3). */
double gint_weight(const gint_handle *h);

/* Static message for a status code. */
const char *gint_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GINT_H */
