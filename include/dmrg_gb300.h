/*
 * dmrg_gb300.h -- C ABI of the GB300 (sm_103a) two-site QC-DMRG hot path.
 *
 * Method: J. Brabec et al., "Massively parallel quantum chemical density
 * matrix renormalization group method" (arXiv:2001.04890).  Section and
 * equation names below are the paper's.
 *
 * The library owns every block operator, task list and Davidson workspace on
 * the GPU.  Callers pass plain host or device pointers and sizes; nothing in
 * this interface is a framework type.  All functions return DMRG_OK (0) or a
 * negative status and then set a thread-local message (dmrg_last_error).  No
 * function aborts the process or traps the GPU; device-side waits are bounded
 * and report DMRG_ETIMEOUT.
 *
 * Conventions shared by every entry point
 *   Orbitals (sites) 0..L-1 in lattice order.  Site basis {0, up, dn, updn}
 *   with |updn> = a+_up a+_dn |0> (Eq. creation_ops read in its stated order).
 *   Jordan-Wigner order: sites in lattice order, up before dn on a site.
 *   Hamiltonian (Eq. H2q) in spin-orbital form
 *       H = sum_pq h_pq a+_ps a_qs + 1/2 sum_pqrs (pq|rs) a+_ps a+_rt a_st a_qs,
 *   h row-major L*L symmetric, v row-major L^4 chemists' (pq|rs), no core energy.
 *   Position k (0 <= k <= L-2): left block l = sites 0..k-1, left site k,
 *   right site k+1, right block r = sites k+2..L-1 (Sec. 2.1, Fig. dmrg_blocks).
 *   Block sectors: (n_up, n_dn) sorted ascending (Sec. 2.1, U(1) symmetry).
 *   psi (Eqs. wf, wf_sec): blocks (a, b, c, d) = (left-block sector, left-site
 *   state, right-site state, right-block sector) with particle numbers adding
 *   to (N_up, N_dn), ordered lexicographically; each block m_a x m_d row-major.
 *   Enlarged left block l (x) s (Eq. renorm): sectors sorted; inside a sector
 *   the (a, b) sub-blocks in lexicographic order, each m_a rows.  Enlarged
 *   right block s (x) r: (c, d) sub-blocks in lexicographic order, m_d rows.
 *   A renormalization matrix O is given per enlarged sector E as a row-major
 *   dim_E x kept_E matrix with orthonormal columns; all sectors concatenated.
 */
#ifndef DMRG_GB300_H
#define DMRG_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DMRG_OK = 0,
  DMRG_EINVAL = -1,   /* bad argument or state-independent precondition   */
  DMRG_ENOMEM = -2,   /* device or host allocation failed                  */
  DMRG_ECUDA = -3,    /* a CUDA or library call failed (message has it)     */
  DMRG_ENOCONV = -4,  /* Davidson hit max_iter before the tolerance          */
  DMRG_ESTATE = -5,   /* call not valid in the current context state        */
  DMRG_ETIMEOUT = -6  /* a bounded device-side wait ran out                  */
};

/* FP64: every operation in FP64.  FP32: FP64 block operators, renormalization and
 * density matrices; FP32 copies of the operators for the Davidson matvecs (FP32
 * CUDA-core arithmetic).  BF16X3: FP64 block operators, renormalization and
 * density matrices; H.psi output blocks with both sides <= 128 and one side >=
 * tc_min (33 by default, 1 routes every such block; see dmrg_set_tune) run on
 * the tcgen05 tensor cores as three-pass split-BF16 products with FP32
 * accumulation in tensor memory, their operand tiles split straight from the
 * FP64 operators (no FP32 copies are held), and the remaining blocks run in
 * FP64.  In both mixed modes Davidson finishes with a defect-corrected
 * refinement that applies H in FP64 to the current vector (see dmrg_davidson),
 * so energies are FP64 quality. */
enum { DMRG_PREC_FP64 = 0, DMRG_PREC_FP32 = 1, DMRG_PREC_BF16X3 = 2 };

typedef struct dmrg_ctx dmrg_ctx; /* opaque, library-owned */

/* Thread-local text of the last error (never NULL; empty if none). */
const char *dmrg_last_error(void);

/*
 * dmrg_init -- problem setup (Sec. 2.1, Eq. H2q; Sec. 2.2 task lists).
 * Copies h (L*L) and v (L^4) from HOST memory.  N electrons, two_sz = N_up - N_dn.
 * M: bond dimension (kept states per block, Eq. renorm).  precision: DMRG_PREC_*.
 * cuda_stream: a cudaStream_t (may be NULL for the legacy default stream);
 * every device operation of this context is ordered on it.
 * Builds the site operators, the deterministic Aufbau product state (orbitals
 * 0..N_up-1 carry an up electron, 0..N_dn-1 a dn electron) and all right
 * blocks of that state, and leaves the context at position 0.
 * Errors: DMRG_EINVAL for L < 2, N outside [0, 2L], |two_sz| > N, parity of N
 * and two_sz different, N_up or N_dn > L, M < 1, non-finite h or v, h not
 * symmetric within 1e-12; DMRG_ENOMEM / DMRG_ECUDA from the device.
 * *out receives the context (owned by the caller until dmrg_free).
 */
int dmrg_init(int L, int N, int two_sz, const double *h, const double *v, int M, int precision,
              void *cuda_stream, dmrg_ctx **out);

/* Release every device and host resource of the context (NULL is allowed). */
int dmrg_free(dmrg_ctx *ctx);

/*
 * dmrg_set_position -- move to two-site position k (0 <= k <= L-2) without
 * changing any block; direction +1 (forward) or -1 (backward) only records
 * the sweep direction.  Blocks needed by later calls must already exist.
 */
int dmrg_set_position(dmrg_ctx *ctx, int k, int direction);

/* Current position k and the recorded sweep direction (+1 / -1); host ints, each may be
 * NULL.  DMRG_EINVAL for a NULL context. */
int dmrg_get_position(dmrg_ctx *ctx, int *k, int *direction);

/*
 * dmrg_psi_layout -- the psi block list of Eq. wf_sec at the current position.
 * If blocks is non-NULL it must hold 7 * (*nblocks from a previous call) ints:
 * per block (a, b, c, d, rows m_a, cols m_d, element offset).  *dim = length of psi.
 * Any output pointer may be NULL.  DMRG_ESTATE if a block is missing.
 */
int dmrg_psi_layout(dmrg_ctx *ctx, int *nblocks, int *blocks, long long *dim);

/*
 * dmrg_block_sectors -- sectors of the left (side 0) or right (side 1) block
 * at the current position: per sector (n_up, n_dn, dim), 3 ints each.
 */
int dmrg_block_sectors(dmrg_ctx *ctx, int side, int *nsec, int *sectors);

/*
 * dmrg_enlarged_layout -- enlarged sectors of l (x) s_l (direction +1) or
 * s_r (x) r (direction -1) at the current position: per sector (n_up, n_dn, dim).
 */
int dmrg_enlarged_layout(dmrg_ctx *ctx, int direction, int *nsec, int *sectors);

/*
 * dmrg_hpsi -- sigma = H psi at the current position (Sec. 2.2.1, Eq. dgemm):
 *   sigma^{s'} = sum_{alpha, s} f(s) A_l^{(alpha,s,s')} psi^s (A_r^{(alpha,s,s')})^T
 * psi and sigma have the dmrg_psi_layout layout and length dim.  If device_ptrs
 * is non-zero both are device pointers valid on the context's stream (sigma
 * is written, not accumulated; psi is not modified; they must not overlap);
 * otherwise both are host pointers and the call copies in and out.  The
 * operators are those of the working precision (FP32 copies in DMRG_PREC_FP32).
 * The result is bitwise repeatable run to run (fixed summation order).
 */
int dmrg_hpsi(dmrg_ctx *ctx, const double *psi, double *sigma, int device_ptrs);

/*
 * dmrg_hpsi_noalloc -- dmrg_hpsi with device pointers that allocates no device
 * memory (no paper counterpart: an interface for callers that cannot allocate,
 * e.g. applications that reserve their whole device-memory budget up front, or
 * latency-critical code that must not block on the CUDA allocator).
 * psi and sigma are device pointers on the context's stream (same layout and
 * semantics as dmrg_hpsi).  The task list of the current position must already
 * exist (any dmrg_hpsi, dmrg_hpsi_flops or dmrg_davidson call at this
 * position builds it), else DMRG_ESTATE.  The chunk partials of the split
 * task list go to one fixed device array of dmrg_hpsi_noalloc_capacity()
 * doubles (16 MiB) that the library holds on every GPU it is loaded on until
 * exit; positions that need more return DMRG_EINVAL with the size needed.
 * The first call on a device looks up that array's device address (a CUDA
 * runtime call); make it before any stream capture.  The array is shared by
 * all calls and contexts in the process and keeps the last call's contents;
 * each call clears the part it uses.  Calls that overlap on the GPU race on
 * it: order them on one stream.  The call does not synchronize, so a
 * tensor-core completion wait that runs out in it (DMRG_PREC_BF16X3) is not
 * seen on return: dmrg_check_status reports it (DMRG_ETIMEOUT), as does the
 * next synchronizing call on the context; the call clears any such report
 * left by an earlier call first, so a report always belongs to the calls
 * made since.
 */
int dmrg_hpsi_noalloc(dmrg_ctx *ctx, const double *psi, double *sigma);
long long dmrg_hpsi_noalloc_capacity(void);

/*
 * dmrg_check_status -- waits for the work queued on the context's stream and
 * reports whether a bounded device-side wait of that work ran out:
 * DMRG_ETIMEOUT (the results of those calls are invalid; the message names the
 * wait) or DMRG_OK.  The report is cleared once read.  Needed only after calls
 * that do not synchronize (dmrg_hpsi_noalloc); every other call checks on its
 * own before it returns.  No paper counterpart (error reporting).
 */
int dmrg_check_status(dmrg_ctx *ctx);

/* Algorithmic FLOPs of one dmrg_hpsi at the current position (host-counted from the task list). */
int dmrg_hpsi_flops(dmrg_ctx *ctx, double *flops, long long *tasks);

/*
 * dmrg_set_psi / dmrg_get_psi -- the context's current wave function in the
 * dmrg_psi_layout layout.  device_ptr != 0: psi is a device pointer (copied on
 * the context stream); 0: a host pointer (the call returns after the copy).
 * dmrg_set_psi also makes it the Davidson starting vector.  dmrg_get_psi
 * returns DMRG_ESTATE if no wave function is held at this position.
 */
int dmrg_set_psi(dmrg_ctx *ctx, const double *psi, int device_ptr);
int dmrg_get_psi(dmrg_ctx *ctx, double *psi, int device_ptr);

/*
 * dmrg_davidson -- lowest eigenpair of Eq. h_mat at the current position by
 * Davidson's method (Sec. 2.2.1); vectors, orthogonalisation, the subspace
 * eigenproblem and residuals are FP64 on the GPU.  In the mixed precisions the
 * matvecs use the low-precision operators until the residual reaches 1e-6 |E|
 * (FP32) or 1e-4 |E| (BF16X3); then each refinement step applies H in FP64 to
 * the current vector (exact residual and Rayleigh quotient) and expands the
 * subspace with low-precision matvecs only, to tol; if the exact residual stops
 * improving, plain FP64 Davidson finishes.  *iters counts all H.psi
 * applications (dmrg_stats separates the low-precision ones).  Diagonal preconditioner
 * (E - diag H)^-1 with |denominator| >= 1e-8, subspace <= 24, thick restart
 * with 2 vectors, converged when ||H psi - E psi|| <= tol for normalized psi.
 * Starts from the current psi when one is set, else from a fixed pseudo-random
 * vector; a fixed seeded admixture of relative size ~6e-4 is added to the
 * start vector, because a state carried over from the previous position lies
 * in one symmetry subspace of H (spin, spin flip) that an FP64 Krylov space
 * never leaves, while the lowest state may lie in another.  *energy, *iters
 * (host; may be NULL).  DMRG_ENOCONV if max_iter is reached (energy and psi
 * still hold the last Ritz pair).
 */
int dmrg_davidson(dmrg_ctx *ctx, double tol, int max_iter, double *energy, int *iters);

/*
 * dmrg_davidson_lowp -- the first phase of dmrg_davidson alone: Davidson with
 * every matvec in the context's working precision (FP32 operators or split-BF16
 * x3 tensor-core products in the mixed precisions, FP64 otherwise) until
 * ||H psi - E psi|| <= tol or max_iter iterations, without the FP64
 * refinement (the residual is that of the low-precision operator).  Vectors,
 * subspace and residuals are FP64 as in dmrg_davidson.  For measurements of
 * the working-precision iteration and for cheap warm-up iterations.  *energy,
 * *iters (host; may be NULL): the Ritz value and the number of H.psi
 * applications (the start vector's included).  DMRG_ENOCONV if max_iter is
 * reached.
 */
int dmrg_davidson_lowp(dmrg_ctx *ctx, double tol, int max_iter, double *energy, int *iters);

/*
 * dmrg_set_davidson -- refinement variant of the mixed-precision Davidson
 * (dmrg_davidson): refine_keep = 0 (default) restarts every refinement step
 * from the current Ritz vector alone; refine_keep = m (1..8) also carries the
 * next m Ritz vectors of the step's subspace, with their low-precision images,
 * into the next step (a thick restart; their couplings to x are taken from
 * the exact H x).  A replica of the algorithm needed far fewer matvecs on
 * spectra with a dense bottom; not yet measured on a GPU.  No effect in
 * DMRG_PREC_FP64.  sweep_max_iter: the matvec cap of every Davidson step of
 * dmrg_sweep / dmrg_sweep_record (default 200).  DMRG_EINVAL for a NULL
 * context, refine_keep outside 0..8 or sweep_max_iter < 1.
 */
int dmrg_set_davidson(dmrg_ctx *ctx, int refine_keep, int sweep_max_iter);

/*
 * dmrg_set_renorm_precision -- arithmetic of the renormalization products
 * O^T (sum of block op (x) site op) O of Eq. renorm_mat (Sec. 2.2.2), in every
 * later dmrg_renormalize and sweep step: DMRG_PREC_FP64 (default) or
 * DMRG_PREC_FP32 (O and the old block's operators rounded to FP32 in the
 * products, FP32 accumulation within each chunk of products, FP64 result and
 * FP64 sums across chunks).  The density matrix, its eigenvectors and the
 * truncation stay FP64.  Independent of the working precision of H.psi.
 * DMRG_EINVAL for a NULL context or another precision.
 */
int dmrg_set_renorm_precision(dmrg_ctx *ctx, int precision);

/*
 * dmrg_renormalize -- truncate the enlarged block and renormalize its
 * operators (Eqs. renorm, renorm_mat; Sec. 2.2.2), then move one position.
 * direction +1: new left block l' = l (x) s_l, position k -> k+1.
 * direction -1: new right block r' = s_r (x) r, position k -> k-1.
 * If O is NULL the basis is the kept eigenvectors of rho^L = psi psi^T
 * (rho^R = psi^T psi) of the current psi: the M largest eigenvalues over all
 * sectors (or the per-direction limits of dmrg_set_bond_dims), ties broken by
 * (sector order, in-sector order), eigenvalues
 * <= 1e-13 never kept; where the M-th and the next eigenvalue differ by less
 * than 1e-10 the cut moves down past that near-degenerate cluster (unless
 * nothing would remain), so the kept space is unique; kept (may be NULL)
 * receives the per-sector counts.
 * Otherwise kept (host, one int per enlarged sector) and O (host, layout in
 * the header comment) define the new basis; the caller guarantees
 * orthonormal columns.  *discarded_weight (may be NULL) = trace(rho) - kept
 * eigenvalues (0 when O is given).  After the move the current psi is
 * transformed into the new position's basis (wave-function prediction) when
 * O was NULL; otherwise it is cleared.
 */
int dmrg_renormalize(dmrg_ctx *ctx, int direction, const int *kept, const double *O,
                     double *discarded_weight);

/*
 * dmrg_truncation_stats -- record of the density-matrix truncations
 * (dmrg_renormalize with O NULL, and the steps of dmrg_sweep) since dmrg_init.
 * The gap of one truncation is the smallest kept eigenvalue minus the largest
 * eigenvalue above 1e-13 that was cut (+infinity when no such eigenvalue was
 * cut).  The cut is moved below near-degenerate clusters (see
 * dmrg_renormalize), so a gap below 1e-10 remains only where the top cluster
 * alone holds more than M states: the kept space, and the energies after it,
 * then depend on rounding (the paper's rule names no order for equal
 * eigenvalues).  Outputs (host, each may be NULL): the last gap, the smallest
 * gap, the number of truncations and the number with gap < 1e-10.  Errors:
 * DMRG_EINVAL (NULL context).
 */
int dmrg_truncation_stats(dmrg_ctx *ctx, double *last_gap, double *min_gap, long long *truncations,
                          long long *straddled);

/*
 * dmrg_block_basis -- export the renormalization matrix O of a stored block
 * (Eq. renorm): the MPS tensor of the block's outermost site (Sec. 2.1, the
 * MPS matrices are the reshaped renormalization matrices).  side 0: the left
 * block of `sites` sites (0..sites-1), made from the left block of sites-1
 * sites and site sites-1; side 1: the right block of `sites` sites
 * (L-sites..L-1), made from site L-sites and the right block of sites-1 sites.
 * Same format as the input of dmrg_renormalize: per enlarged sector (in the
 * enlarged-layout order of the header comment) the kept count, and O as the
 * concatenated row-major dim_E x kept_E matrices.  Outputs (host, each may be
 * NULL): *nsec enlarged sectors, kept (nsec ints), O (*nO doubles), *nO.
 * Chaining the exported O of blocks 1..n rebuilds the block's basis states
 * in the product basis of its sites.  Errors: DMRG_EINVAL (bad arguments),
 * DMRG_ESTATE (no stored basis for that block, e.g. never built or released).
 */
int dmrg_block_basis(dmrg_ctx *ctx, int side, int sites, int *nsec, int *kept, double *O, long long *nO);

/*
 * dmrg_orbital_entropies -- one- and two-orbital entropies of the current
 * two-site wave function (Eq. wf_sec) at its two sites k and k+1.  The
 * two-orbital reduced density matrix over the site-state pairs (b, c) of the
 * two sites, rho[(b c), (b' c')] = sum_{a,d} <psi_{a b c d}, psi_{a b' c' d}>
 * (trace = |psi|^2), is built on the host from a copy of psi; the one-orbital
 * matrices are its partial traces (diagonal in {0, up, dn, updn}).  s3 (may
 * be NULL) receives the von Neumann entropies -tr(r ln r) of the
 * trace-normalised matrices {s_k, s_{k+1}, s_{k,k+1}}; the mutual information
 * of the pair is s_k + s_{k+1} - s_{k,k+1}.  rho2 (may be NULL): the 16 x 16
 * matrix, row-major over 4 b + c, site states in the order 0, up, dn, updn.
 * The paper uses these entropies for orbital ordering (single-site entropies
 * and mutual information, Sec. 3) without defining them; these are the
 * standard definitions.  Errors: DMRG_EINVAL (NULL context or both outputs
 * NULL), DMRG_ESTATE (no wave function at this position), DMRG_ECUDA.
 */
int dmrg_orbital_entropies(dmrg_ctx *ctx, double *s3, double *rho2);

/*
 * dmrg_mutual_information -- one-orbital entropies of every orbital and the
 * mutual information I_ij = s_i + s_j - s_ij of every orbital pair (the
 * quantities Sec. 3 uses to order the orbitals), from the wave function at
 * position 0 and the right blocks of every length as stored (one backward
 * pass, e.g. dmrg_sweep, which ends at position 0; run dmrg_davidson there
 * first for the converged state).  Each right block state is a column of its
 * renormalization matrix over (site state) x (next right block state) with
 * orthonormal columns, so the two-orbital reduced density matrix of orbitals
 * i < j follows by carrying a density matrix with orbital i's states open
 * through the sites between them (each traced; an element that changes the
 * parity of orbital i picks up (-1)^(particles) of each, the Jordan-Wigner
 * string of moving orbital j next to orbital i) and tracing everything right
 * of j.  Host arithmetic on copies of psi and the renormalization matrices,
 * O(L^2) transfers of sector-blocked matrices.  Outputs (host, each may be
 * NULL, not all): I (L*L, row-major, symmetric, zero diagonal), s1 (L
 * entropies), rho_pairs (L*L*256: the 16 x 16 matrix of pair (i, j), i < j, at
 * (i*L + j)*256, rows and columns 4 b + c with b, c the site states of i and
 * j in the order 0, up, dn, updn; other entries 0).  Errors: DMRG_EINVAL,
 * DMRG_ESTATE (not at position 0, no wave function, or a right block missing
 * or released).
 */
int dmrg_mutual_information(dmrg_ctx *ctx, double *I, double *s1, double *rho_pairs);

/*
 * dmrg_sweep -- nsweeps two-site sweeps (Sec. 2.1, Fig. dmrg_blocks): forward
 * over positions 0..L-3 (Davidson then dmrg_renormalize(+1)), backward over
 * L-2..1 (Davidson then dmrg_renormalize(-1)).  Starts from position 0 in the
 * forward direction.  energies (host, may be NULL) receives one energy per
 * Davidson step: nsweeps * 2 * (L - 2) values.  Each step runs Davidson to tol
 * with at most 200 matvecs (dmrg_set_davidson changes the cap); a step that
 * does not converge keeps its last Ritz
 * pair and the sweep goes on.  Errors: DMRG_EINVAL (NULL context, nsweeps < 0,
 * tol <= 0, L < 3), else those of dmrg_davidson and dmrg_renormalize.
 */
int dmrg_sweep(dmrg_ctx *ctx, int nsweeps, double tol, double *energies);

/*
 * dmrg_sweep_record -- dmrg_sweep with per-step records (each output host,
 * may be NULL, one slot per Davidson step in sweep order): energies, the
 * discarded weight of the step's truncation (dmrg_renormalize), and entropies
 * (3 per step: one-orbital entropies of the step's two sites k, k+1 and
 * their two-orbital entropy, as dmrg_orbital_entropies after the step's
 * Davidson).  Over one sweep every site and every adjacent pair appears.
 */
int dmrg_sweep_record(dmrg_ctx *ctx, int nsweeps, double tol, double *energies, double *discarded,
                      double *entropies);

/*
 * dmrg_set_bond_dims -- asymmetric bond dimensions: later RDM truncations of
 * dmrg_renormalize keep at most m_forward states in new left blocks
 * (direction +1) and m_backward in new right blocks (direction -1), e.g. the
 * larger M on the enlarged half and the smaller on the environment of the
 * paper's largest case.  dmrg_init sets both to M.  DMRG_EINVAL if either < 1.
 */
int dmrg_set_bond_dims(dmrg_ctx *ctx, int m_forward, int m_backward);

/*
 * dmrg_set_precision -- change the working precision of the Davidson matvecs
 * (DMRG_PREC_*) of an existing context; blocks and the wave function are kept,
 * the old precision's low-precision operator copies, tensor-core tiles and task
 * list are released at once (so the largest workloads can switch without
 * holding both), and the H.psi task lists are rebuilt on next use.
 * DMRG_EINVAL for an unknown precision.  Synchronizes the stream.
 */
int dmrg_set_precision(dmrg_ctx *ctx, int precision);

/*
 * dmrg_release_block -- free the stored block of `sites` sites on side 0 (left)
 * or 1 (right) to bound device memory when only part of a sweep is needed (the
 * paper keeps every block for later sweeps; this is a memory option).  A later
 * position that needs a released block fails with DMRG_ESTATE until it is
 * rebuilt by renormalization; wave-function prediction across a released block
 * is skipped.  DMRG_EINVAL for a block the current position uses, a side other
 * than 0/1 or sites outside 1..L-2; releasing an absent block is a no-op.
 * Synchronizes the context stream.
 */
int dmrg_release_block(dmrg_ctx *ctx, int side, int sites);

/*
 * dmrg_block_op -- introspection of one stored operator of the left (side 0)
 * or right (side 1) block at the current position, in its family layout:
 * for each ket sector a with a bra sector a' in order, the m_a' x m_a block.
 * kind: 0 H, 1 a+_i, 2 T_i (left blocks), 3 V_i (right blocks), 4 a+_i a+_j,
 * 5 a+_i a_j (spin-orbital indices 2*site + spin).  out (host) may be NULL to
 * query *n (element count).  DMRG_EINVAL if the block stores no such operator.
 */
int dmrg_block_op(dmrg_ctx *ctx, int side, int kind, int i, int j, double *out, long long *n);

/*
 * Batched independent instances (many problems of uneven L and M, e.g. one per
 * integral set): the H.psi task lists of n contexts, each at its current
 * position, run as one task list over concatenated psi / sigma vectors; every
 * kernel class is one grouped launch for all instances, captured once into a
 * CUDA graph and replayed (Sec. 2.2.1 task list, merged over instances).
 * All contexts must share one stream and the same precision class; they must
 * not change position while the batch lives.  dmrg_batch_layout gives the n+1
 * offsets of each instance's psi in the concatenated vector (dmrg_psi_layout
 * order inside) and the summed algorithmic FLOPs of one batched H.psi.
 * dmrg_batch_hpsi: psi and sigma of the concatenated length, device pointers
 * on the shared stream (device_ptrs != 0) or host pointers (copied in and
 * out); sigma is written, not accumulated.  The batch does not own the
 * contexts: free the batch first.  Errors: DMRG_EINVAL (n < 1, NULL
 * arguments, contexts on different streams or precision classes),
 * DMRG_ESTATE (a context without the blocks of its position; from
 * dmrg_batch_hpsi: a context whose H.psi task list was rebuilt or released
 * since the batch was built, by a move, a precision or launch-shape change:
 * the batch addresses that context's operator copies and must be created
 * again),
 * DMRG_ETIMEOUT (a bounded tensor-core wait ran out; that call's sigma is
 * invalid), DMRG_ENOMEM / DMRG_ECUDA.
 */
typedef struct dmrg_batch dmrg_batch;
int dmrg_batch_create(int n, dmrg_ctx *const *ctxs, dmrg_batch **out);
int dmrg_batch_layout(dmrg_batch *batch, long long *offsets, double *flops);
int dmrg_batch_hpsi(dmrg_batch *batch, const double *psi, double *sigma, int device_ptrs);
int dmrg_batch_free(dmrg_batch *batch);

/*
 * Launch-shape autotuning of the H.psi task list (the grouped launch of the
 * sector-pair products of Sec. 2.2.1, Eq. dgemm; the paper has no counterpart:
 * its task sizes are fixed by the MPI distribution).  Six parameters shape a
 * task list: target_chunks (the work of all output blocks is cut into about
 * this many equal-work chunks), min_chunk (no chunk lighter than this many
 * FLOPs), tc_min (output blocks with a side >= tc_min and both sides <= 128
 * run on the tensor-core kernel in DMRG_PREC_BF16X3), by_work (1: chunks
 * launched heaviest first; 0: in output-block order), flat_wide (1: the
 * kernel for blocks of at most 32 x 32 runs one wide CTA per SM, 0: two
 * narrower CTAs per SM) and tc_tiny (the tensor-core kernel's shape: 1 = every
 * block with m <= 64 and q and every task's p <= 32 runs on the 32-column
 * shape, five CTAs per SM, in a launch of its own; 0 = that shape only when
 * every block fits it, else the 64- and 128-row shapes).  Defaults: 8192, 2e5,
 * 33, 0, 1, 0.
 *
 * dmrg_autotune builds candidate task lists for the current position, times
 * `reps` complete H.psi launch sequences of each (CUDA events, on a seeded
 * vector; synchronizes the stream), keeps the fastest for this and later
 * positions and rebuilds the position's task lists with it.  best_ms (may be
 * NULL) receives the time of one H.psi with the chosen shape; params (may be
 * NULL, 6 doubles) the chosen target_chunks, min_chunk, tc_min, by_work,
 * flat_wide, tc_tiny.  Results of
 * H.psi differ between shapes only by floating-point summation order.
 * Errors: DMRG_EINVAL (NULL context, reps < 1), DMRG_ESTATE (blocks of the
 * position not built), DMRG_ETIMEOUT, DMRG_ECUDA.
 * dmrg_set_tune sets the parameters without timing (DMRG_EINVAL unless
 * target_chunks >= 1, min_chunk >= 0, 1 <= tc_min <= 129, by_work,
 * flat_wide and tc_tiny 0 or 1); the task lists are rebuilt on next use.
 * dmrg_get_tune writes the current six parameters.
 * dmrg_batch_autotune does the same for a batch (every context still at the
 * position it had at dmrg_batch_create, else DMRG_ESTATE); the CUDA graph of
 * the batch is captured again on the next dmrg_batch_hpsi.
 */
int dmrg_autotune(dmrg_ctx *ctx, int reps, double *best_ms, double *params);
int dmrg_set_tune(dmrg_ctx *ctx, double target_chunks, double min_chunk, int tc_min, int by_work,
                  int flat_wide, int tc_tiny);
int dmrg_get_tune(dmrg_ctx *ctx, double *params);
int dmrg_batch_autotune(dmrg_batch *batch, int reps, double *best_ms, double *params);

/*
 * dmrg_stats -- counters since context creation or the last reset (host outputs,
 * any may be NULL): total device time of the H.psi kernel launches (CUDA events
 * recorded on the context stream around each launch), number of H.psi calls,
 * their summed algorithmic FLOPs, kernels launched by this library in the
 * process, Davidson iterations (all, and those with low-precision matvecs),
 * and the residual norm of the last Davidson run.  reset != 0 zeroes the
 * counters afterwards.  Synchronizes the context stream.
 */
int dmrg_stats(dmrg_ctx *ctx, int reset, double *hpsi_ms, long long *hpsi_calls, double *hpsi_flops,
               long long *kernel_launches, long long *davidson_iters, long long *davidson_iters_lowp,
               double *last_residual);

/*
 * dmrg_plan_hpsi_flops -- host only (no GPU): algorithmic FLOPs and task count
 * of one H.psi at position k for given block sector tables (per sector
 * n_up, n_dn, dim; nl left and nr right sectors, sorted), i.e. what
 * dmrg_hpsi_flops reports for blocks with those sectors.
 */
int dmrg_plan_hpsi_flops(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                         const int *sec_l, int nr, const int *sec_r, double *flops, long long *tasks);

/*
 * dmrg_selftest_tcgen05 -- device check of the library's tensor-core encodings
 * (diagnostic): C (128 x N) = A (128 x K) B^T (B is N x K), inputs rounded to
 * bf16, FP32 accumulation in tensor memory.  Host pointers, row-major.
 * N in 16..256 and K in 16..64, multiples of 16.  DMRG_ETIMEOUT if the
 * bounded completion wait ran out.
 */
int dmrg_selftest_tcgen05(int N, int K, const float *A, const float *B, float *C);

/*
 * dmrg_debug_set_wait_limit -- fault detection test hook (no paper
 * counterpart), process-wide.  Sets the number of polls of every pipeline wait
 * of the tensor-core kernel (a job's operands landed, a stage freed, T or D
 * complete) for launches made from now on; tries < 0 restores the default
 * (2^22 polls).  When a wait runs out the kernel records the time-out, lets
 * its copies and MMAs in flight finish (those drain waits keep the default
 * limit), releases its tensor memory and returns, and the call reports
 * DMRG_ETIMEOUT; the context stays usable.  tries = 0 makes every pipeline
 * wait give up at once, before any copy or MMA is issued.  Always DMRG_OK.
 */
int dmrg_debug_set_wait_limit(long long tries);

/*
 * dmrg_debug_fail_alloc -- fault injection on the host (no paper
 * counterpart), process-wide: for n > 0, the n-th device allocation of the
 * library from now fails as if the device were out of memory, so the call
 * making it returns DMRG_ENOMEM; later allocations succeed.  n <= 0 disarms.
 * Always DMRG_OK.
 */
int dmrg_debug_fail_alloc(long long n);

/*
 * dmrg_debug_tasks -- host-only dump of the H.psi task list the planner builds
 * for the same arguments as dmrg_plan_hpsi_flops: per task 7 ints (output psi
 * block index, m, n, p, q, identity flags (1: left identity, 2: right
 * identity), element offset of the input psi block), in build order
 * (grouped = 0) or grouped by output block as the GPU task list runs it
 * (grouped = 1).  out may be NULL to query *ntasks; DMRG_EINVAL if
 * cap < *ntasks.  No GPU is used.
 */
int dmrg_debug_tasks(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                     const int *sec_l, int nr, const int *sec_r, int grouped, int *out, long long cap,
                     long long *ntasks);

/*
 * dmrg_debug_exec -- host-only dump of the execution plan the GPU runs for the
 * H.psi task list of dmrg_debug_tasks (the grouped products of Eq. dgemm,
 * Sec. 2.2.1): each output block's tasks in their cheaper association, cut
 * into chunks of about equal work that accumulate into scratch slots, then an
 * ordered reduction of the slots into sigma.  tensor_cores: 1 routes blocks to
 * the tensor-core kernel as DMRG_PREC_BF16X3 does; tune: NULL (defaults) or 5
 * doubles target_chunks, min_chunk, tc_min, by_work, tc_tiny as in
 * dmrg_set_tune.
 * counts (8): execution entries, chunks of the 32 x 32 tile kernel, of the
 * flattened-lane kernel, of the tensor-core kernel, reduction groups, tiles,
 * scratch elements, reduced elements.  Optional arrays (NULL to skip; sizes
 * from counts): xs_out 8 per entry (psi offset of Y, n, p, Y row stride, Y
 * column stride, identity flags, X offset, Z offset; -1 for identity),
 * grp_out 8 per chunk (kernel 0/1/2, slot offset, slot row stride, slot column
 * stride, m, q, first entry, entry count), red_out 8 per output block (first
 * reduced element, first slot offset, sigma offset, row stride, column stride,
 * m, q, chunk count).  Operator offsets are relative to each arena.
 */
int dmrg_debug_exec(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                    const int *sec_l, int nr, const int *sec_r, int tensor_cores, const double *tune,
                    long long *counts, long long *xs_out, long long *grp_out, long long *red_out);

/*
 * dmrg_debug_validate -- host-only bounds check of the execution plan that
 * dmrg_debug_exec describes (tune: NULL for the default launch shape, or 5
 * doubles as in dmrg_debug_exec).  The four operand arenas
 * (stored operators and pre-summed temporaries of both blocks) are given
 * distinct element bases, so every operand address names its arena.  Every
 * operand view of every chunk (rows x columns with its strides) must lie
 * inside its arena, every psi view inside psi, every chunk slot and every
 * reduction inside the scratch array, identity sides must be square; with
 * tensor_cores, every operator and psi tile's source view inside its arena or
 * psi, every tile inside the tile arenas, every task's X, Y^T and Z^T tile
 * reads and its stack inside their bounds, every output slot inside the
 * scratch array.
 * *checked receives the number of views and slots checked, *bad the number
 * of violations (the first one is described in dmrg_last_error).  No GPU is
 * used.
 */
int dmrg_debug_validate(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                        const int *sec_l, int nr, const int *sec_r, int tensor_cores, const double *tune,
                        long long *checked, long long *bad);

/*
 * dmrg_debug_tc -- host-only dump of the tensor-core launch plan for the same
 * task list as dmrg_debug_exec with tensor_cores = 1 (FP32 operand addresses):
 * the blocks routed to the tensor cores, ordered by kernel shape, their tasks
 * grouped into stacks that share a psi block, and the operator and psi tiles
 * in order of first use.  tune: NULL or 5 doubles as in dmrg_debug_exec.
 * counts (9): tasks, blocks, operator tiles, psi tiles, operator tile bytes,
 * psi tile bytes, blocks of the 64 x 32, 64 x 64 and 128 x 128 shapes.
 * Optional arrays (NULL to skip): te_out 14 per task (X tile, Y^T tile, Z^T
 * tile byte offsets, stack length or 0, execution-list entry, X offset, X row
 * and column strides, Z offset, Z row and column strides, psi offset of Y, n,
 * p), tg_out 7 per block (output offset, row stride, column stride, m, q,
 * first task, task count), ts_out 6 per operator tile (source element offset
 * times 4 or -1 for identity, tile byte offset, source row and column strides,
 * rows, columns), ps_out 4 per psi tile (psi offset, tile byte offset, n, p).
 * No GPU is used.
 */
int dmrg_debug_tc(int L, int N, int two_sz, const double *h, const double *v, int k, int nl, const int *sec_l,
                  int nr, const int *sec_r, const double *tune, long long *counts, long long *te_out,
                  long long *tg_out, long long *ts_out, long long *ps_out);

/*
 * dmrg_debug_pair_rdm -- host-only form of dmrg_orbital_entropies for a
 * caller's two-site wave function: nblocks blocks, abcd 4 ints per block
 * (left block sector, left site state 0..3, right site state 0..3, right block
 * sector; sectors are any integer labels), off_size 2 per block (element
 * offset in psi, element count m_a m_d), psi the values.  rho2 (256, may be
 * NULL) and s3 (3, may be NULL) as in dmrg_orbital_entropies.  DMRG_EINVAL on
 * bad arguments or blocks of one (a, d) pair with different sizes.  No GPU is
 * used.
 */
int dmrg_debug_pair_rdm(int nblocks, const int *abcd, const long long *off_size, const double *psi,
                        double *rho2, double *s3);

/* Planner introspection (host only, no GPU): text dumps of the H pieces at
 * position k and of the blocking definitions of a new block's operators. */
int dmrg_debug_pieces(int L, const double *h, const double *v, int k, int l_empty, int r_empty,
                      int compress, char *buf, long long buflen, long long *needed);
int dmrg_debug_newops(int L, const double *h, const double *v, int k, int side, int old_empty,
                      char *buf, long long buflen, long long *needed);

/*
 * dmrg_debug_truncation -- host-only run of the truncation rule that
 * dmrg_renormalize applies to the density-matrix spectrum (Sec. 2.1): the
 * mkeep largest eigenvalues over all sectors, ties by (sector, in-sector rank
 * from the top), eigenvalues <= 1e-13 never kept, the cut moved below a
 * near-degenerate cluster (consecutive eigenvalues closer than 1e-10) that
 * straddles it unless nothing would remain.  In: nsectors, dims (one
 * int per sector), ev_ascending (sum of dims doubles: each sector's spectrum in
 * ascending order, sectors concatenated).  Out: kept (one int per sector),
 * cols (may be NULL; sum of kept ints: per sector, the kept columns as indices
 * into the ascending order, largest eigenvalue first), out3 = {trace, kept
 * weight, cut gap as in dmrg_truncation_stats}.  DMRG_EINVAL on bad arguments.
 * No GPU is used.
 */
int dmrg_debug_truncation(int nsectors, const int *dims, const double *ev_ascending, int mkeep,
                          int *kept, int *cols, double *out3);

#ifdef __cplusplus
}
#endif
#endif /* DMRG_GB300_H */
