// One step of the hierarchical Markov chain (Sec. 5, the three-step
// algorithm; Eq. 4step steps 0, 1 and 3):
//   U0 <- U;
//   n_inner times, per colour pass: U' <- proposal(U) on the active links
//     (heat-bath / over-relaxation), block filter of (U, U') restoring the
//     rejected blocks (with one level of recursion: filter of the
//     sub-blocks, then the blocks' Schur filter, Eq. 4step steps 1-2), U <- U';
//   stochastic estimate of det(D'^dag D' / D^dag D) for (U0, U) with n_global
//   interpolation factors, global accept; U <- U0 on rejection.
// Random-stream counters: step << 20 | iteration << 4 | colour pass for the
// proposal and filter of an iteration, step << 20 | n_inner << 4 for the
// global step.  Every operation is asynchronous on the handle's stream, so a
// step can be captured into a CUDA graph (dd_graph_begin) and replayed with
// the counters advanced by (step << 20).
#include "dd_internal.h"

extern "C" int dd_chain_step(dd_t h, void* U, const dd_chain_params* p, const dd_chain_buffers* b,
                             unsigned long long step) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (!U || !p || !b || !b->U0 || !b->Up || !b->ln_b || !b->acc_b || !b->ln_g || !b->acc_g || !b->margin)
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_chain_step: null argument");
    if (p->n_inner < 0 || p->n_block < 1 || p->n_global < 1 || p->n_hb < 0 || p->n_or < 0 || p->n_schur < 0 ||
        p->gauge_fix_sweeps < 0 ||
        (p->colour_passes != 1 && p->colour_passes != 2) || step >= (1ull << 40))
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_chain_step: bad parameters");
    if (h->has_sub && p->n_schur > 0 && (!b->ln_bs || !b->acc_bs))
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_chain_step: step 2 needs ln_bs and acc_bs");
    // the recursive hierarchy updates all active links of the sub-blocks at
    // once, which decouples them only for the PAPER / INNER6 sets
    if (h->has_sub && (p->colour_passes != 1 || h->active_mode == DD_ACTIVE_INTRA))
        return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_chain_step: recursion needs one colour pass and PAPER/INNER6 links");
    const size_t bytes = (size_t)h->g.V * 4 * 9 * 16;
    DD_CUDA(h, cudaMemcpyAsync(b->U0, U, bytes, cudaMemcpyDeviceToDevice, h->stream));
    for (int it = 0; it < p->n_inner; ++it) {
        for (int pass = 0; pass < p->colour_passes; ++pass) {
            const int colour_mask = p->colour_passes == 2 ? pass + 1 : 3;
            const uint64_t ctr = (step << 20) | ((uint64_t)it << 4) | (uint64_t)pass;
            DD_CUDA(h, cudaMemcpyAsync(b->Up, U, bytes, cudaMemcpyDeviceToDevice, h->stream));
            rc = dd_gauge_update(h, b->Up, colour_mask, p->beta, p->n_hb, p->n_or, p->seed, ctr);
            if (rc) return rc;
            rc = dd_block_filter(h, U, b->Up, colour_mask, p->filter_mode, p->n_block, p->seed, ctr, b->ln_b,
                                 b->acc_b);
            if (rc) return rc;
            if (h->has_sub && p->n_schur > 0) {
                // step 2: the blocks' Schur complements of their sub-blocks
                rc = dd_block_schur_filter(h, U, b->Up, colour_mask, p->n_schur, p->seed, ctr, b->ln_bs, b->acc_bs);
                if (rc) return rc;
            }
            DD_CUDA(h, cudaMemcpyAsync(U, b->Up, bytes, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    const uint64_t ctr = (step << 20) | ((uint64_t)p->n_inner << 4);
    if (p->gauge_fix_sweeps > 0) {
        // the same ratio for the proposal fixed relative to U0 (Sec. 4)
        DD_CUDA(h, cudaMemcpyAsync(b->Up, U, bytes, cudaMemcpyDeviceToDevice, h->stream));
        rc = dd_relative_gauge_fix(h, b->U0, b->Up, p->gauge_fix_sweeps, nullptr);
        if (rc) return rc;
        rc = dd_det_ratio_estimate(h, b->U0, b->Up, p->n_global, p->seed, ctr, DD_EST_FACTORS | DD_EST_INTERP_ALL,
                                   b->ln_g);
    } else {
        rc = dd_det_ratio_estimate(h, b->U0, U, p->n_global, p->seed, ctr, DD_EST_FACTORS, b->ln_g);
    }
    if (rc) return rc;
    return dd_global_accept(h, U, b->U0, b->ln_g, p->n_global, p->seed, ctr, b->acc_g, b->margin);
}
