/*
 * dd.h - C ABI of the GB300 (sm_103a) library for the domain-decomposed
 * Wilson-Dirac hot path of the hierarchical acceptance algorithm of
 * Leder, Finkenrath, Knechtli, "Fermions as global correction in lattice QCD"
 * (Lattice 2011).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Lattice: extents L0 x L1 x L2 x L3, axis 3 is time, canonical site index
 *   s = x0 + L0*(x1 + L1*(x2 + L2*x3)).  Every extent must be even.  Blocks
 *   (domains) of extent b_a tile the lattice from the origin; the number of
 *   blocks per direction must be even and >= 2 (checkerboard colouring of the
 *   blocks, Sec. 3 and Fig. 1); block colour = (sum_a B_a) mod 2, 0 = black.
 * Fields at the boundary are FP64 complex numbers stored as interleaved
 *   (re, im) doubles, canonical site order:
 *     gauge field  U[s][a][i][j]   72 doubles per site: SU(3) link from s to
 *                                  s + a-hat (a = lattice axis 0..3);
 *     spinor       psi[s][spin][c] 24 doubles per site (4 spins x 3 colours),
 *                                  chiral gamma basis (gamma_0 = time =
 *                                  axis 3, gamma_5 = diag(1, 1, -1, -1));
 *     nrhs spinors are stored one after another (stride 24*V doubles), or
 *     24*V/2 doubles for even-site vectors (DD_OP_DTILDE*, DD_OP_HEO).
 *   Pointers named U, in, out, x, b, eta are DEVICE pointers owned by the
 *   caller; the library never frees them.  Scalars written through pointers
 *   documented as "device" are valid after the handle's stream has been
 *   synchronised (dd_sync); "host" pointers are written before return.
 * Operator: D = 1 - kappa*H with the Wilson hopping term
 *   (H psi)(x) = sum_a [(1 - gamma_a) U_a(x) psi(x + a) + (1 + gamma_a) U_a(x - a)^dag psi(x - a)],
 *   hops across the time edge multiplied by bc_time.
 * Random streams: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *   (element, purpose << 24 | sub, ctr mod 2^32, ctr >> 32); Gaussian noise with
 *   density ~ exp(-|eta|^2) by Box-Muller in FP64 (the normalisation for which
 *   the estimator of Sec. 4 is unbiased).
 * Errors: every call returns DD_OK (0) or a negative DD_ERR_* code; nothing is
 *   thrown across the boundary; dd_last_error() gives a message.  Device-side
 *   failures (a solver that hits its iteration cap, a non-finite reduction, a
 *   bounded wait that ran out) set a status word read by dd_status(); no kernel
 *   traps.  All work is enqueued on the stream given to dd_init.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define DD_OK 0
#define DD_ERR_INVALID_ARG (-1)
#define DD_ERR_UNSUPPORTED (-2)
#define DD_ERR_CUDA (-3)
#define DD_ERR_NOT_CONVERGED (-4)
#define DD_ERR_NUMERIC (-5)
#define DD_ERR_TIMEOUT (-6)
#define DD_ERR_NO_WORKSPACE (-7)

/* arithmetic / storage precision of a kernel */
#define DD_PREC_F64 0 /* FP64 storage and arithmetic */
#define DD_PREC_F32 1 /* FP32 storage (links: rows 1-2, third row rebuilt), FP32 arithmetic */
#define DD_PREC_F16 2 /* FP16 storage (spinors with a per-site FP32 scale), FP32 arithmetic */
#define DD_PREC_DF64 3 /* dd_params.outer_prec only: double-float (pairs of FP32, 48-bit significand)
                          arithmetic on FP64-sized storage */

/* active-link sets (Sec. 3: links with at most one end on a block boundary) */
#define DD_ACTIVE_AUTO 0   /* INTRA if a block extent <= 2, INNER6 if all >= 8, else PAPER */
#define DD_ACTIVE_PAPER 1  /* the rule applied to the block itself */
#define DD_ACTIVE_INNER6 2 /* the rule applied to the block shrunk by one site per side */
#define DD_ACTIVE_INTRA 3  /* every link with both ends in one block (updated colour by colour) */
#define DD_ACTIVE_ALL 4    /* every link: pure-gauge updates of the whole lattice (thermalisation);
                              not a decoupled set for the block filter */

/* operators of dd_apply_D */
#define DD_OP_D 0          /* D psi on the whole lattice */
#define DD_OP_DDAG 1       /* D^dag psi = gamma5 D gamma5 psi */
#define DD_OP_DTILDE 2     /* even sites: (1 - kappa^2 H_eo H_oe) psi_e */
#define DD_OP_DTILDE_DAG 3 /* even sites: gamma5 Dtilde gamma5 psi_e */
#define DD_OP_HEO 4        /* even sites <- odd sites: H_eo psi_o (in: odd-site vector) */
#define DD_OP_INTER 5      /* (D_bw + D_wb) psi: only the hops that cross block faces */

/* purposes of the random stream (counter word 1, bits 24-31) */
#define DD_PURPOSE_GLOBAL_NOISE 1
#define DD_PURPOSE_BLOCK_NOISE 2
#define DD_PURPOSE_HEATBATH 3
#define DD_PURPOSE_BLOCK_ACCEPT 5
#define DD_PURPOSE_GLOBAL_ACCEPT 6
#define DD_PURPOSE_USER_NOISE 7
#define DD_PURPOSE_BLOCK_SCHUR_NOISE 4  /* step 2 of Eq. 4step (dd_block_schur_filter) */
#define DD_PURPOSE_BLOCK_SCHUR_ACCEPT 8

/* estimator modes (Eq. param) */
#define DD_EST_FACTORS 0  /* factor i uses U_i, U_{i+1} of the geodesic path, its own eta_i */
#define DD_EST_REPLICAS 1 /* every factor uses (U, U'), its own eta_i (variance measurement) */
#define DD_EST_INTERP_ALL 4 /* flag: interpolate every link that differs between U and U' (after a
                               relative gauge fixing), not only the active links */

/* block filter modes (Eq. 4step, step 1) */
#define DD_FILTER_STOCHASTIC 0
#define DD_FILTER_EXACT 1

typedef struct dd_handle* dd_t;

typedef struct {
    int dims[4];       /* lattice extents, axis 3 = time */
    int block[4];      /* block (domain) extents */
    double kappa;      /* hopping parameter of D = 1 - kappa*H */
    int bc_time;       /* fermion boundary phase in time: -1 antiperiodic, +1 periodic */
    int active_mode;   /* DD_ACTIVE_* */
    int max_rhs;       /* largest nrhs or number of factors of any later call */
    int inner_prec;    /* precision of the inner global solver: DD_PREC_F64/F32/F16 */
    int block_prec;    /* precision of the inner block solver: DD_PREC_F64/F32 */
    double tol_global; /* true relative residual of global solves, ||b - D x|| / ||b|| */
    double tol_block;  /* true relative residual of Dirichlet block solves */
    double tol_inner;  /* residual reduction asked of one inner solve (defect correction) */
    int maxit;         /* iteration cap of any single Krylov solve */
    int features;      /* workspace parts to plan: DD_FEAT_* bits, 0 = all */
    int krylov;        /* inner Krylov method of mixed-precision solves: DD_KRYLOV_* */
    int sub_block[4];  /* one level of recursive decomposition (Eq. ddrec): sub-block
                          extents, each block split into an even number of sub-blocks
                          per direction; all 0 = no recursion.  With sub-blocks the
                          active links are those of the sub-blocks (active_mode applied
                          to the sub-blocks; dd_chain_step needs PAPER or INNER6),
                          dd_block_filter acts on the sub-blocks (Eq. 4step step 1)
                          and dd_block_schur_filter on the blocks (step 2). */
    int outer_prec;    /* arithmetic of the true residual r = b - D x in the defect-correction
                          loop of mixed-precision solves (Sec. 5): DD_PREC_F64 (default, 0) or
                          DD_PREC_DF64 (double-float: every operation on the FP32 pipe, rounding
                          error about 2^-47 of the summed term magnitudes; the workspace then
                          holds one more FP64-sized copy of each gauge-field slot) */
    int sap_ncy;       /* DD_KRYLOV_SAP_GCR: Schwarz cycles per preconditioner application (default 4, 1..16) */
    int sap_nmr;       /* DD_KRYLOV_SAP_GCR: BiCGStab iterations per approximate block solve (default 4, 1..64) */
    int sap_nkv;       /* DD_KRYLOV_SAP_GCR: directions kept by the flexible GCR before a restart (default 6, at most 16) */
} dd_params;

/* inner Krylov method of the FP32/FP16 solves (the FP64 solver is always CGNR) */
#define DD_KRYLOV_CGNR 0     /* CG on the even-odd normal equations Dtilde^dag Dtilde */
#define DD_KRYLOV_BICGSTAB 1 /* BiCGStab on Dtilde (van der Vorst), restarted by the FP64 loop */
/* Global solves by flexible GCR on the whole operator D, preconditioned with
 * sap_ncy cycles of the Schwarz alternating procedure over the black/white
 * blocks (the domain-decomposition solver the block decomposition of Sec. 3
 * comes from): per cycle and colour the residual of that colour's blocks and
 * an approximate solve of every such block (sap_nmr BiCGStab iterations of
 * its even-odd Dirichlet system).  The inner system Dtilde e = r of the FP64
 * defect correction is solved as D (e, e_o) = (r, 0), whose even part is e.
 * FP32 arithmetic, hop inputs and links in the inner precision (F16 or F32);
 * Dirichlet solves (Schur pieces, filter) use BiCGStab.  Eager calls only
 * (the GCR polls its residuals from the host): inside a graph capture the
 * global solve returns DD_ERR_UNSUPPORTED; outer_prec must be DD_PREC_F64. */
#define DD_KRYLOV_SAP_GCR 2

/* workspace features (dd_params.features); entry points that need a part the
 * workspace was not planned with fail with DD_ERR_UNSUPPORTED */
#define DD_FEAT_SOLVE 1    /* dd_apply_D, dd_apply_D_block, dd_solve */
#define DD_FEAT_ESTIMATE 2 /* dd_det_ratio_estimate, dd_block_filter (stochastic), dd_interpolate-based paths */
#define DD_FEAT_EXACT 4    /* dd_logdet_exact, exact block filter */

/* Fill p with defaults: kappa 0.125, bc_time -1, DD_ACTIVE_AUTO, max_rhs 1,
 * inner F16, block F32, tol_global 1e-10, tol_block 1e-12, tol_inner 1e-3,
 * maxit 20000, krylov CGNR, sap_ncy 4, sap_nmr 4, sap_nkv 6.  dims/block are
 * zeroed and must be set by the caller. */
int dd_default_params(dd_params* p);

/* Create a handle for one lattice and block decomposition (Sec. 3, Eq. domdec).
 * stream: a cudaStream_t (NULL = legacy default stream); all later work of
 * the handle is enqueued on it.  Builds the geometry tables on the host and
 * uploads them (the only allocation the library makes itself).
 * Errors: DD_ERR_INVALID_ARG for odd or non-dividing extents, blocks per
 * direction odd or < 2, kappa <= 0, max_rhs < 1, an unknown precision or
 * active mode, more than 2^30 sites; DD_ERR_UNSUPPORTED when 12 V >= 2^32
 * (the noise streams number the spinor components of site s as 12 s + k in
 * one 32-bit counter word, which would wrap); DD_ERR_CUDA on a CUDA error. */
int dd_init(dd_t* h, const dd_params* p, void* stream);

/* Bytes of device workspace the handle needs for its max_rhs. */
int dd_workspace_size(dd_t h, size_t* bytes);

/* Hand the library device memory of at least dd_workspace_size bytes,
 * 256-byte aligned.  The caller owns it and must keep it alive until
 * dd_finalize or the next dd_set_workspace.  Every entry point below except
 * dd_get_maps and dd_status fails with DD_ERR_NO_WORKSPACE before this call. */
int dd_set_workspace(dd_t h, void* dev_ptr, size_t bytes);

/* Copy the geometry tables to HOST arrays (any pointer may be NULL):
 *   nbr[s*8 + 2a]     = canonical index of s + a-hat, nbr[s*8 + 2a + 1] = of s - a-hat;
 *   sign[s*8 + k]     = fermion phase of that hop (+1 or bc_time);
 *   dd_order[q]       = canonical site at block-ordered position q (black
 *                       blocks first in increasing block id, then white;
 *                       sites of a block in local lexicographic order, Sec. 3);
 *   block_of[s]       = block id of s (lexicographic in block coordinates);
 *   active[s*4 + a]   = 1 if link (s, a) belongs to the active set.
 * Sizes: V = L0*L1*L2*L3. */
int dd_get_maps(dd_t h, int32_t* nbr, int32_t* sign, int32_t* dd_order, int32_t* block_of, uint8_t* active);

/* out = op(U) in for nrhs spinors (op = DD_OP_*), in precision prec
 * (the FP32/FP16 forms round links and spinors to that storage first).
 * Definition: the Wilson-Dirac operator (Sec. 5: the unimproved Wilson-Dirac operator), its
 * even-odd Schur complement and the block-interaction terms of Eq. domdec.
 * in/out: device, canonical spinors (even-site vectors for DTILDE/DTILDE_DAG,
 * odd-site in / even-site out for HEO; the sites of one parity in canonical
 * order).  in and out must not overlap. */
int dd_apply_D(dd_t h, void* out, const void* in, const void* U, int op, int prec, int nrhs);

/* out = D_b psi on the blocks of the colours in colour_mask (bit 0 black,
 * bit 1 white), 0 on the other sites: every hop that leaves a block is
 * dropped (Dirichlet block operators, D_bb and D_ww of Eq. domdec). */
int dd_apply_D_block(dd_t h, void* out, const void* in, const void* U, int colour_mask, int prec, int nrhs);

/* Solve D x = b for nrhs right-hand sides (shared U) by CG on the even-odd
 * normal equations; with prec = DD_PREC_F32/F16 the inner solver runs in that
 * precision inside an FP64 defect-correction loop whose residual is the FP64
 * true residual ||b - D x|| / ||b|| <= tol_global.  iters (host, may be NULL)
 * receives the total inner iterations, relres (host, nrhs doubles, may be
 * NULL) the final true relative residuals.  DD_ERR_NOT_CONVERGED if maxit was
 * reached first (x then holds the last iterate). */
int dd_solve(dd_t h, void* x, const void* b, const void* U, int nrhs, int prec, int* iters, double* relres);

/* The Schwarz preconditioner of DD_KRYLOV_SAP_GCR alone: out = sap_ncy
 * cycles of the Schwarz alternating procedure over the black/white blocks
 * (Sec. 3 decomposition; per cycle black blocks, then white blocks, each
 * after the residual rho - D z of its sites is formed) applied to in, from
 * z = 0, with approximate block solves of sap_nmr BiCGStab iterations in
 * the precision prec (DD_PREC_F32 or DD_PREC_F16).  With exact block solves
 * one cycle is the block Gauss-Seidel step z = [[A, 0], [C, E]]^{-1} rho.
 * in, out: device canonical FP64 spinors (nrhs of them, 24 V doubles each);
 * U: device canonical FP64 gauge field.  The handle must have been created
 * with krylov DD_KRYLOV_SAP_GCR (else DD_ERR_UNSUPPORTED) and an even block
 * extent along axis 0. */
int dd_sap_apply(dd_t h, void* out, const void* in, const void* U, int nrhs, int prec);

/* Complex Gaussian noise (density ~ exp(-|eta|^2), Sec. 4) on every site for
 * nrhs vectors: component (s, spin, c) of vector r uses element
 * s*12 + spin*3 + c, purpose `purpose`, sub = r, counter ctr, key seed. */
int dd_noise(dd_t h, void* eta, int nrhs, int purpose, uint64_t seed, uint64_t ctr);

/* U_t = U (U^dag U')^t, t = i/n, on the active links (other links copied from
 * U); the geodesic path of Eq. param with the branch for which det = 1
 * (phases in (-pi, pi], the largest lowered / smallest raised by 2 pi when
 * they sum to +-2 pi).  i = 0 gives U and i = n gives U' exactly. */
int dd_interpolate(dd_t h, void* U_t, const void* U, const void* U_new, int i, int n);

/* Stochastic estimate of the global Schur-complement step (Eq. 4step step 3,
 * Sec. 4): n factors, factor i with M_i = Dhat[U_{i+1}]^{-1} Dhat[U_i]
 * (DD_EST_FACTORS; U_0 = U_old, U_n = U_new) or M = Dhat[U_new]^{-1} Dhat[U_old]
 * (DD_EST_REPLICAS), noise eta_i on the black sites (purpose
 * DD_PURPOSE_GLOBAL_NOISE, sub = i).  ln_out[i] (device, n doubles) receives
 * -eta_i^dag (M_i^dag M_i - 1) eta_i, computed as -(2 Re<eta, d> + |d|^2) with
 * d = (M_i - 1) eta_i, d = [D'^{-1} (s, 0)]_black,
 * s = B'E'^{-1}C' eta - A'A^{-1}BE^{-1}C eta.  Block solves to tol_block,
 * the global solve to tol_global in inner_prec. */
int dd_det_ratio_estimate(dd_t h, const void* U_old, const void* U_new, int n, uint64_t seed, uint64_t ctr,
                          int mode, double* ln_out);

/* Block filter (Eq. 4step step 1; Sec. 5, acceptance block by block): for every
 * block of a colour in colour_mask, ln_b[block] (device, nblocks doubles) =
 * sum over n factors of -(2 Re<eta, d> + |d|^2), d = D_b[U_{i+1}]^{-1}
 * (D_b[U_i] - D_b[U_{i+1}]) eta_{b,i} (DD_FILTER_STOCHASTIC, purpose
 * DD_PURPOSE_BLOCK_NOISE, sub = i), or 2 (ln|det D_b[U_new]| - ln|det D_b[U_old]|)
 * (DD_FILTER_EXACT, dense LU, blocks of at most 256 sites).  Then accept[block]
 * (device, nblocks bytes) = ln u_b < ln_b (u_b: purpose DD_PURPOSE_BLOCK_ACCEPT,
 * element = block id), 1 for blocks outside colour_mask, and the active links
 * of rejected blocks are copied back from U_old into U_new (in place).
 * All (block, factor) solves run in one persistent launch. */
int dd_block_filter(dd_t h, const void* U_old, void* U_new, int colour_mask, int mode, int n, uint64_t seed,
                    uint64_t ctr, double* ln_b, uint8_t* accept);

/* Block Schur filter, step 2 of Eq. 4step with one level of recursion
 * (Eq. ddrec; handles created with sub_block set): for every block b of the
 * colours in colour_mask the stochastic estimate of
 * ln det(Dhat_b'^dag Dhat_b' / Dhat_b^dag Dhat_b), Dhat_b = the Schur
 * complement of the block operator D_b with respect to its sub-blocks,
 * summed over n interpolation factors (Eq. param, one eta per factor):
 *   ln_b[b] = -sum_i sum_{x in b} (2 Re<eta_i, delta_i>_x + |delta_i|_x^2),
 *   delta_i = [D1[U_{i+1}]^{-1} (s_i, 0)]_black,
 *   s_i = B'E'^{-1}C' eta_i - A'A^{-1}BE^{-1}C eta_i,
 * with D1 the Dirichlet operator of the blocks, A/E the sub-block operators
 * of the black/white sub-blocks and B/C the hops across sub-block faces
 * inside a block (unprimed: U_i, primed: U_{i+1}); eta_i on the black
 * sub-blocks (purpose DD_PURPOSE_BLOCK_SCHUR_NOISE, element 12 s + 3 spin
 * + colour, sub = i).  Solves: sub-block Dirichlet solves to tol_block, the
 * block Dirichlet solve to tol_global (mixed precision as dd_solve).
 * accept[b] = ln u_b < ln_b[b] (purpose DD_PURPOSE_BLOCK_SCHUR_ACCEPT,
 * element b; 1 for unselected colours); the active links of rejected blocks
 * are restored from U_old in U_new.  ln_b (nblocks doubles) and accept
 * (nblocks bytes) are device arrays over the blocks (not the sub-blocks).
 * DD_ERR_UNSUPPORTED without sub-blocks. */
int dd_block_schur_filter(dd_t h, const void* U_old, void* U_new, int colour_mask, int n, uint64_t seed,
                          uint64_t ctr, double* ln_b, uint8_t* accept);

/* Relative gauge fixing (Sec. 4: reduces the variance of the eigenvalue
 * distribution of M^dag M; the paper does not state the method): U_new is
 * replaced in place by U_new^g, g(x) in SU(3), g_a(x) U_new_a(x) g(x+a)^dag,
 * with g raising F[g] = sum_{x,a} Re tr(U_a(x)^dag g(x) U_new_a(x) g(x+a)^dag)
 * from g = 1 by `sweeps` sweeps (sites of even, then odd parity; at each site
 * one Cabibbo-Marinari pass over the SU(2) subgroups (0,1), (1,2), (0,2)
 * maximising Re tr(g W) with W the sum of the eight link products through
 * the site).  Determinant ratios are unchanged (gauge invariance); the fixed
 * field differs from U on more than the active links, so its estimate needs
 * DD_EST_INTERP_ALL.  functional (device, 1 double, may be NULL) receives
 * F at the final g.  U, U_new: device gauge fields. */
int dd_relative_gauge_fix(dd_t h, const void* U, void* U_new, int sweeps, double* functional);

/* The block filter of several lattices at once (Eq. 4step step 1): every
 * (block, factor) solve of all nh handles runs in ONE persistent launch, the
 * items of the largest blocks first; blocks may differ in shape between the
 * lattices (e.g. 4^4, 6^4 and 8^4).  Per handle k the results are those of
 * dd_block_filter(hs[k], U_old[k], U_new[k], colour_mask, DD_FILTER_STOCHASTIC,
 * n, seed, ctr, ln_b[k], accept[k]) (same random streams, same arithmetic).
 * All handles must have been created on one stream and share the block
 * precision; every launch of the call goes to the first handle's stream, so
 * a CUDA graph recorded on hs[0] (dd_graph_begin; no other handle of the
 * batch may be recording) holds the whole batch (the descriptor tables must
 * then equal those of the last eager call with the same ws).
 * DD_ERR_INVALID_ARG otherwise.  hs, U_old,
 * U_new, ln_b and accept are host arrays of nh pointers (the pointers
 * themselves device memory).  ws: device memory of at least
 * dd_block_filter_batch_workspace(nh, hs, n) bytes, 256-byte aligned, owned
 * by the caller (holds the item queue and the thread-block scratch slots). */
int dd_block_filter_batch_workspace(int nh, const dd_t* hs, int n, size_t* bytes);
int dd_block_filter_batch(int nh, const dd_t* hs, const void* const* U_old, void* const* U_new, int colour_mask,
                          int n, uint64_t seed, uint64_t ctr, double* const* ln_b, uint8_t* const* accept, void* ws,
                          size_t ws_bytes);

/* Proposal (Eq. 4step step 0): n_hb Cabibbo-Marinari heat-bath sweeps of the
 * Wilson plaquette action at beta, each followed by n_or over-relaxation
 * sweeps, on the active links of the blocks of the colours in colour_mask,
 * in place.  Sweep order: direction 0..3, site parity even then odd;
 * subgroups (0,1), (1,2), (0,2); Kennedy-Pendleton sampler with at most 64
 * tries (after which the subgroup element is kept; counted in dd_status).
 * Random numbers: purpose DD_PURPOSE_HEATBATH, element 4*s + a,
 * sub = sweep << 16 | subgroup << 12 | draw. */
int dd_gauge_update(dd_t h, void* U, int colour_mask, double beta, int n_hb, int n_or, uint64_t seed, uint64_t ctr);

/* Global acceptance (Eq. 4step step 3 decision): accept iff
 * ln u < sum_i ln_r[i] (ln_r device, n doubles; u: purpose
 * DD_PURPOSE_GLOBAL_ACCEPT, element 0).  On rejection U_old is copied into U.
 * accept (device, 1 byte) receives the decision, ln_margin (device, 1 double,
 * may be NULL) the value sum_i ln_r[i] - ln u. */
int dd_global_accept(dd_t h, void* U, const void* U_old, const double* ln_r, int n, uint64_t seed, uint64_t ctr,
                     uint8_t* accept, double* ln_margin);

/* Exact check path (Sec. 3: the block determinants are obtained exactly from
 * an LU factorisation): dense FP64 LU with partial pivoting of D (which = 0,
 * out[0] = ln|det D|, lattices of at most 512 sites) or of every block
 * operator D_b (which = 1, out[b] = ln|det D_b|, blocks of at most 256 sites),
 * or of the domain Schur complement Dhat (which = 2, out[0] = ln|det Dhat|,
 * at most 512 sites).  out: device doubles.  Blocked LU (panels of 32
 * columns); panels of matrices above 384 rows are factorised by one
 * cooperative launch whose thread blocks meet at a bounded grid barrier.
 * Device status (dd_status): DD_ERR_NUMERIC for a zero pivot,
 * DD_ERR_TIMEOUT if a grid barrier gave up waiting (the results are then
 * invalid). */
int dd_logdet_exact(dd_t h, const void* U, int which, double* out);

/* Trailing update of the dense LU of dd_logdet_exact (matrices above 384
 * rows) and the product B E^-1 C of its Schur-complement assembly (which =
 * 2): on = 1 (default) on the FP16 tensor cores with FP64 accuracy by the
 * Ozaki scheme (every FP64 row and column scaled by a power of two and cut
 * into 8 integer slices of 7 bits; the 36 slice pairs of the 8 heaviest
 * weights multiplied with mma.sync, whose FP32 accumulation is exact for
 * these integers, grouped exactly in int64 and summed in FP64; what is left
 * out stays below the
 * rounding bound of an FP64 dot product); on = 0 on the FP64 FMA pipe (no
 * counterpart in the paper: the tensor-core form of its exact check path).
 * Falls back to FP64 FMA when the exact-path workspace has no room for the
 * slices.  Errors: DD_ERR_INVALID_ARG (on not 0 or 1). */
int dd_lu_tensor_cores(dd_t h, int on);

/* Check of the bounded wait in the grid barrier of the LU panel launch (the
 * paper has no counterpart: failure detection of the only kernel of the
 * library that waits on other thread blocks).  Runs a cooperative launch of
 * up to 8 thread blocks through three grid barriers; with missing > 0 the
 * last barrier waits for that many arrivals that never come, gives up after
 * its poll limit (a few seconds), raises DD_ERR_TIMEOUT in the device status
 * word (dd_status) and returns.  *passed = 1 when every block passed all
 * barriers, else 0.  Synchronises the handle's stream; needs the exact-path
 * workspace (DD_FEAT_EXACT).  Errors: DD_ERR_INVALID_ARG (passed NULL,
 * missing outside 0..64), DD_ERR_UNSUPPORTED, DD_ERR_CUDA. */
int dd_barrier_check(dd_t h, int missing, int* passed);

/* Mean plaquette <Re tr U_P / 3> (device, 1 double). */
int dd_plaquette(dd_t h, const void* U, double* out);

/* Wait for the handle's stream. */
int dd_sync(dd_t h);

/* Read and clear the device status word: 0, or a DD_ERR_* code raised by a
 * kernel since the last call.  heatbath_fails (may be NULL) receives the
 * number of subgroup updates left unchanged by the Kennedy-Pendleton cap. */
int dd_status(dd_t h, int* device_status, long long* heatbath_fails);

/* Message of the last error of this handle (static storage, never NULL). */
const char* dd_last_error(dd_t h);

/* Instrumentation (no counterpart in the paper).  dd_launch_count: kernels
 * the handle has launched since dd_init (host, written before return).
 * dd_kernel_timer: CUDA-event timing, on the handle's stream, of the
 * even-odd hop kernel of one kind (0: FP16 in / FP16 out, 1: FP16 in / FP32
 * out with the xpay term, 2: FP64, 3: double-float residual hops).  op 1 = reset and start timing every
 * `every`-th launch of each kind, op 0 = stop, op 2 = synchronise the stream
 * and return the summed duration (ms), the number of timed launches and the
 * output sites those launches processed (systems already converged in a
 * batch are skipped and not counted) for `kind`; host pointers, may be NULL.
 * Event recording adds well under a microsecond per timed launch. */
int dd_launch_count(dd_t h, long long* launches);
int dd_kernel_timer(dd_t h, int op, int kind, int every, double* total_ms, long long* timed, long long* sites);
/* Timer kinds beyond the whole-lattice hops 0-3: 4 FP64, 5 FP16 -> FP16 and
 * 6 FP16 -> FP32 hops restricted to the blocks on the sites of one block
 * colour (Dirichlet solves of the Schur pieces; kind 4 also the filter);
 * 7 the persistent block solver (sites = block items of the timed
 * launches); 8 FP16 -> FP16 and 9 FP16 -> FP32 hops restricted to the
 * blocks over every site (the whole-lattice filter form). */
#define DD_TIMER_KIND_COUNT 10

/* Iteration counts of the solves since the last dd_kernel_timer(op 1) (the
 * paper has no counterpart: work accounting for the measurement).  kind 0:
 * whole-lattice defect-correction solves (dd_solve, the global step); 1:
 * Dirichlet solves restricted to the blocks (Schur pieces, whole-lattice
 * filter form); 2: the persistent block solver.  out (host, 5 long long):
 * kinds 0-1: batched solves, systems (right-hand sides) solved, inner Krylov
 * iterations summed over systems, outer (defect-correction) cycles summed
 * over the batched solves, sites x inner iterations; kind 2: launches, block
 * items, inner iterations summed over items, outer cycles summed over items,
 * block sites x inner iterations.  Kinds 0-1 count eager (polled) solves
 * only; kind 2 synchronises the stream. */
int dd_solver_stats(dd_t h, int kind, long long* out);

/* Arithmetic peaks of the current GPU, measured (the paper has no
 * counterpart: roofline denominators of the ALU-bound kernels).  Fills
 * tflops[0] FP64 FMA, [1] FP32 FMA, [2] FP64 mma.sync m8n8k4 (tensor core)
 * throughput in TFLOP/s: 8 thread blocks of 256 threads per SM, eight
 * independent chains per thread, best of three CUDA-event timed launches on
 * `stream`.  Allocates and frees one small device buffer; takes well under a
 * second.  Returns DD_OK, DD_ERR_INVALID_ARG (tflops NULL) or DD_ERR_CUDA. */
int dd_alu_peaks(double* tflops, void* stream);

/* The block filter of Eq. 4step step 1 in two parts, for a filter whose
 * blocks are shared out among several GPUs (the blocks decouple because the
 * active links of different blocks share no plaquette, Sec. 3):
 * dd_block_ratios_range computes the stochastic log-ratios (n factors, as
 * dd_block_filter with DD_FILTER_STOCHASTIC in its persistent per-block form,
 * same random streams) of the blocks at block-order positions
 * [pos0, pos0 + npos) (black blocks occupy positions 0 .. nblocks/2 - 1,
 * white blocks the rest); ln_b (device, nblocks doubles, by block id) gets
 * them, and 0 for every other block.  Summing the ln_b of disjoint ranges
 * that cover the selected colours gives dd_block_filter's ln_b bit for bit.
 * dd_block_accept then takes decisions from a complete ln_b (ln u_b < ln_b,
 * u_b from DD_PURPOSE_BLOCK_ACCEPT keyed by block id; blocks outside
 * colour_mask accepted) into accept (device, nblocks bytes) and restores
 * U_old on the active links of rejected blocks of U_new (in place).
 * Errors: DD_ERR_INVALID_ARG for a range outside [0, nblocks), n outside
 * [1, max_rhs] or null pointers. */
int dd_block_ratios_range(dd_t h, const void* U_old, const void* U_new, int pos0, int npos, int n, uint64_t seed,
                          uint64_t ctr, double* ln_b);
int dd_block_accept(dd_t h, const void* U_old, void* U_new, int colour_mask, const double* ln_b, uint64_t seed,
                    uint64_t ctr, uint8_t* accept);

/* Allocation-free block log-ratios (the paper has no counterpart: this is an
 * interface variant for callers that cannot allocate device memory — code
 * running while a CUDA graph is captured in global mode, where cudaMalloc is
 * illegal; plug-ins whose host application owns all device memory; loops that
 * cannot afford the implicit device synchronisation of cudaMalloc/cudaFree).
 * It needs no handle and no workspace and calls no allocating routine.
 * Computes, for every block of the colours in colour_mask, the one-factor
 * stochastic log-ratio of the block filter,
 *   ln_b[block id] = -(2 Re<eta, d> + |d|^2),  d = D_b[U_new]^{-1} (D_b[U_old] - D_b[U_new]) eta_b,
 * eta_b from purpose DD_PURPOSE_BLOCK_NOISE, sub 0 (the values dd_block_filter
 * gives for n = 1 when U_new differs from U_old only on active links);
 * 0 for the other blocks.  Solver (fixed caps, not the handle settings of
 * dd_block_filter): FP64 defect correction to relative residual tol_block,
 * at most 12 cycles, around an FP32 conjugate-gradient solve of the block's
 * normal equations (relative target 1e-10, at most 2000 iterations per
 * cycle).  dd_block_filter's inner solver is BiCGStab: both reach tol_block,
 * by different iterations.  A block whose refinement does not reach
 * tol_block within the 12 cycles, or whose residual or result is not finite,
 * gets ln_b = NaN (the failure shows in the caller's own output, since the
 * entry point has no handle and no status word).
 * dims/block: host arrays (extents even, blocks per direction even and >= 2);
 * U_old, U_new: device, canonical FP64 gauge fields; ln_b: device, nblocks
 * doubles.  Work is enqueued on `stream` (a cudaStream_t, NULL = default).
 * 12 V >= 2^32 (V = sites): DD_ERR_UNSUPPORTED, as in dd_init.
 * Scratch: one file-scope device array of 64 MiB, held by every GPU that
 * loads the library until the process exits; a block may have at most
 * 64 MiB / 1248 B (about 53000) sites, else DD_ERR_UNSUPPORTED.  The first
 * call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream
 * capture.  Every call shares the array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Returns DD_OK, DD_ERR_INVALID_ARG, DD_ERR_UNSUPPORTED or
 * DD_ERR_CUDA (launch errors only; results are valid after the stream is
 * synchronised). */
int dd_block_ratios_noalloc(const int dims[4], const int block[4], double kappa, int bc_time, int colour_mask,
                            const void* U_old, const void* U_new, uint64_t seed, uint64_t ctr, double tol_block,
                            double* ln_b, void* stream);

/* One step of the hierarchical chain (Sec. 5, the three-step algorithm;
 * Eq. 4step steps 0, 1 and 3), all on the handle's stream:
 *   U0 <- U; n_inner times, per colour pass (colour_passes = 1: both colours
 *   at once; 2: black blocks, then white, for the intra-block active set):
 *   Up <- U, n_hb heat-bath + n_or over-relaxation sweeps on Up, block filter
 *   of (U, Up) with n_block factors (rejected blocks restored), U <- Up;
 *   then the n_global-factor estimate for (U0, U) and the global accept
 *   (U <- U0 on rejection).
 * With sub-blocks (one level of recursion) every iteration runs step 0,
 * step 1 on the sub-blocks and, when n_schur > 0, step 2 on the blocks
 * (dd_block_schur_filter, same counter), before U <- Up.
 * With gauge_fix_sweeps > 0 the global step estimates the ratio for the
 * proposal fixed to U0 (dd_relative_gauge_fix into Up, DD_EST_INTERP_ALL);
 * U itself keeps the unfixed proposal (the ratio is the same).
 * Counters: step << 20 | iteration << 4 | pass for the proposal and filter,
 * step << 20 | n_inner << 4 for the global step (step < 2^40).
 * U: device gauge field, updated in place.  All buffers are caller-owned
 * device memory: U0, Up gauge fields (72 V doubles each); ln_b (nblocks
 * doubles) and acc_b (nblocks bytes) of the last filter; ln_g (n_global
 * doubles), acc_g (1 byte), margin (1 double) of the global step.
 * n_global, n_block <= max_rhs of the handle. */
typedef struct dd_chain_params {
    double beta;
    int n_inner;
    int n_block;
    int n_global;
    int n_hb;
    int n_or;
    int filter_mode;   /* DD_FILTER_STOCHASTIC or DD_FILTER_EXACT */
    int colour_passes; /* 1 or 2 */
    int n_schur;       /* factors of the block Schur filter (step 2; handles with sub-blocks; 0 = skip) */
    uint64_t seed;
    int gauge_fix_sweeps; /* > 0: relative gauge fixing of the proposal before the global estimate */
    int reserved;
} dd_chain_params;
typedef struct dd_chain_buffers {
    void* U0;
    void* Up;
    double* ln_b;      /* step 1: per smallest block (sub-blocks when the handle has them) */
    uint8_t* acc_b;
    double* ln_g;
    uint8_t* acc_g;
    double* margin;
    double* ln_bs;     /* step 2: per block (n_schur > 0 only; else may be NULL) */
    uint8_t* acc_bs;
} dd_chain_buffers;
int dd_chain_step(dd_t h, void* U, const dd_chain_params* p, const dd_chain_buffers* b, unsigned long long step);

/* CUDA-graph capture of library calls (no counterpart in the paper).
 * dd_graph_begin opens a capture: every following call on the handle is
 * recorded, not run, on a private stream of the handle, until dd_graph_end
 * closes it and instantiates the graph (*graph, owned by the caller, freed
 * by dd_graph_destroy).  Solver loops are recorded as conditional WHILE
 * nodes whose stopping rule runs on the device, so a replay needs no host
 * round trip.  Inside a capture: iteration counts and residuals are not
 * written to host pointers; a solve that misses its target or breaks down
 * sets the device status word (dd_status) instead of returning an error;
 * the inner iteration budget of a defect-correction cycle is the full
 * maxit.  Calls whose device tables depend on their arguments (the batched
 * block filter) must have run once eagerly with the same arguments first,
 * else DD_ERR_UNSUPPORTED.
 * dd_graph_launch enqueues one replay on the handle's stream with every
 * random-stream counter of the recorded calls increased by ctr_offset (a
 * device word read by the kernels): a chain step recorded with step 0
 * replays as step k with ctr_offset = k << 20.  Replays reuse the device
 * buffers named at capture time.  dd_graph_nodes: nodes of the top-level
 * graph (host).  Results match eager calls bit for bit. */
typedef struct dd_graph* dd_graph_t;
int dd_graph_begin(dd_t h);
int dd_graph_end(dd_t h, dd_graph_t* graph);
int dd_graph_launch(dd_graph_t graph, unsigned long long ctr_offset);
int dd_graph_nodes(dd_graph_t graph, size_t* nodes);
int dd_graph_destroy(dd_graph_t graph);

/* Autotuner of the launch shapes (no counterpart in the paper).
 * what: DD_TUNE_HOP (thread-block size x sites per thread of the even-odd
 * hop kernels, FP16/FP32 storage and FP64 separately), DD_TUNE_BLOCK
 * (thread-block size and thread blocks per SM of the persistent block
 * solver, at most 4 per SM, and whether the stochastic block filter runs
 * faster as that persistent launch or as batched whole-lattice Dirichlet
 * solves of all blocks, one right-hand side per factor), optionally with
 * DD_TUNE_NO_CACHE.  Each candidate is timed with CUDA events on the
 * handle's stream on this handle's lattice: the hop on zeroed solver
 * vectors (max_rhs right-hand sides), the block solver on one block-filter
 * pass over the fields (U_old, U_new) (device gauge fields; required for
 * DD_TUNE_BLOCK, may be NULL otherwise).  The fastest shape is kept by the
 * handle and used by every later launch.  The result is cached per process
 * and per (device, lattice, blocks, inner precision, max_rhs); when the
 * environment variable DD_TUNE_CACHE names a file, tuned shapes are
 * appended to it and read back by later processes.  report (host, may be
 * NULL) receives the chosen shapes and the average launch times (ms) of the
 * chosen and of the default shapes (0 when taken from the cache).  Runs
 * kernels and synchronises the stream; not allowed inside a capture.
 * dd_set_tuning sets the shapes directly (threads 64 or 128 and 1 or 2
 * sites per thread for the FP16/FP32 hops; 64 or 128 threads and 1 site per
 * thread for the FP64 hops; 64, 128 or 256 threads and 1..4 blocks per SM
 * for the block solver; filter_masked 0 = persistent block-filter launch,
 * 1 = whole-lattice Dirichlet solves).
 * Changing the block-solver shape changes dd_block_filter_batch_workspace. */
#define DD_TUNE_HOP 1
#define DD_TUNE_BLOCK 2
#define DD_TUNE_NO_CACHE 4
typedef struct dd_tune_report {
    int hop_tpb, hop_spt, hop64_tpb, hop64_spt, block_tpb, block_ctas_per_sm;
    int from_cache;
    float hop_ms, hop_default_ms, hop64_ms, hop64_default_ms, block_ms, block_default_ms;
    int filter_masked;      /* 1: the stochastic block filter runs as whole-lattice solves */
    float filter_masked_ms; /* time of that form (one factor) */
} dd_tune_report;
int dd_autotune(dd_t h, int what, const void* U_old, const void* U_new, int reps, dd_tune_report* report);
int dd_set_tuning(dd_t h, int hop_tpb, int hop_spt, int hop64_tpb, int hop64_spt, int block_tpb,
                  int block_ctas_per_sm, int filter_masked);

/* Release the handle's own tables; the workspace stays with the caller. */
int dd_finalize(dd_t h);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
