// One entry point per operation: cos_forward, cos_grad and cos_subsets take a cos_problem
// (lattice, weight kind, precision, input form) and hand it to the implementation of that case.
// The descriptor is validated here; each implementation checks its own sizes and pointers as
// before, so the error behaviour of every case is the one documented in cos.h.
#include <string>

#include "cos_internal.h"

using namespace cosdp;

namespace {

cos_status bad(const char *fn, const char *why) {
    set_error(std::string(fn) + ": " + why);
    return COS_ERR_ARG;
}

// Lattice and weight kind in range; the coordinates form names its tables and vertices.
cos_status check_problem(const cos_problem *p, const char *fn) {
    if (!p) return bad(fn, "null problem");
    if (p->lattice != COS_SQUARE && p->lattice != COS_BIPARTITE) return bad(fn, "unknown lattice");
    if (p->weights != COS_LOOPS && p->weights != COS_DETERMINANTS) return bad(fn, "unknown weight kind");
    if (p->tables && p->weights == COS_LOOPS && p->h_shift)
        return bad(fn, "loop weights from coordinates take their shift weights from the tables (h_shift must be NULL)");
    return COS_OK;
}

}  // namespace

extern "C" cos_status cos_forward(const cos_problem *p, double *d_out, double *d_abs_mass, cos_stream_t s) {
    const char *fn = "cos_forward";
    cos_status st = check_problem(p, fn);
    if (st != COS_OK) return st;
    const bool sq = p->lattice == COS_SQUARE, loops = p->weights == COS_LOOPS;
    if (p->tables) {
        if (sq && loops)
            return cos_connected_sum_batch(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset, p->d_site,
                                           p->d_tau, p->precision, d_out, d_abs_mass, s);
        if (sq)
            return cos_connected_det_batch(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset, p->d_site,
                                           p->d_tau, p->h_shift, p->precision, d_out, d_abs_mass, s);
        if (loops)
            return cos_connected_sum_bipartite_batch(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset,
                                                     p->d_site, p->d_tau, p->precision, d_out, d_abs_mass, s);
        return cos_connected_det_bipartite_batch(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset, p->d_site,
                                                 p->d_tau, p->h_shift, p->precision, d_out, d_abs_mass, s);
    }
    if (sq && loops)
        return cos_connected_sum_matrices(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->n_mat, p->loop_weight,
                                          p->h_shift, p->d_M, p->precision, d_out, d_abs_mass, s);
    if (sq)
        return cos_connected_det_matrices(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->h_shift, p->d_M,
                                          p->precision, d_out, d_abs_mass, s);
    if (loops)
        return cos_connected_sum_bipartite_matrices(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->n_mat,
                                                    p->loop_weight, p->h_shift, p->d_M, p->precision, d_out,
                                                    d_abs_mass, s);
    return cos_connected_det_bipartite_matrices(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->h_shift, p->d_M,
                                                p->precision, d_out, d_abs_mass, s);
}

extern "C" cos_status cos_grad(const cos_problem *p, const double *d_gout, double *d_out, double *d_gM,
                               const int64_t *d_gmoff, double *d_gshift, double *d_gmu, double *d_galpha,
                               cos_stream_t s) {
    const char *fn = "cos_grad";
    cos_status st = check_problem(p, fn);
    if (st != COS_OK) return st;
    if (p->precision != COS_FP64) {
        set_error("cos_grad: gradients are FP64 only");
        return COS_ERR_UNIMPLEMENTED;
    }
    const bool sq = p->lattice == COS_SQUARE, loops = p->weights == COS_LOOPS;
    if (p->tables) {
        if (loops && d_gshift) return bad(fn, "loop weights from coordinates: use d_galpha (d_gshift must be NULL)");
        if (!loops && d_galpha)
            return bad(fn, "determinant weights: the diagonal shifts' gradient is d_gshift (d_galpha must be NULL)");
        if (sq && loops)
            return cos_connected_sum_grad(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset, p->d_site, p->d_tau,
                                          d_gout, d_out, d_gM, d_gmoff, d_gmu, d_galpha, s);
        if (sq)
            return cos_connected_det_grad(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset, p->d_site, p->d_tau,
                                          p->h_shift, d_gout, d_out, d_gM, d_gmoff, d_gmu, d_gshift, s);
        if (loops)
            return cos_connected_sum_bipartite_grad(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset,
                                                    p->d_site, p->d_tau, d_gout, d_out, d_gM, d_gmoff, d_gmu,
                                                    d_galpha, s);
        return cos_connected_det_bipartite_grad(p->tables, p->n_cfg, p->n_max, p->d_order, p->d_offset, p->d_site,
                                                p->d_tau, p->h_shift, d_gout, d_out, d_gM, d_gmoff, d_gmu, d_gshift,
                                                s);
    }
    if (d_gmoff || d_gmu || d_galpha)
        return bad(fn, "explicit matrices: dLoss/dM is written at d_moff; d_gmoff, d_gmu, d_galpha must be NULL");
    if (sq && loops)
        return cos_connected_sum_matrices_grad(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->n_mat, p->loop_weight,
                                               p->h_shift, p->d_M, d_gout, d_out, d_gM, d_gshift, s);
    if (sq)
        return cos_connected_det_matrices_grad(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->h_shift, p->d_M, d_gout,
                                               d_out, d_gM, d_gshift, s);
    if (loops)
        return cos_connected_sum_bipartite_matrices_grad(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->n_mat,
                                                         p->loop_weight, p->h_shift, p->d_M, d_gout, d_out, d_gM,
                                                         d_gshift, s);
    return cos_connected_det_bipartite_matrices_grad(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->h_shift, p->d_M,
                                                     d_gout, d_out, d_gM, d_gshift, s);
}

extern "C" cos_status cos_subsets(const cos_problem *p, int all_roots, double *d_c, double *d_a, cos_stream_t s) {
    const char *fn = "cos_subsets";
    cos_status st = check_problem(p, fn);
    if (st != COS_OK) return st;
    if (p->tables) {
        set_error("cos_subsets: explicit matrices only (gather them with cos_gather / cos_gather_bipartite)");
        return COS_ERR_UNIMPLEMENTED;
    }
    const bool sq = p->lattice == COS_SQUARE, loops = p->weights == COS_LOOPS;
    if (sq && loops)
        return cos_connected_sum_subsets(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->n_mat, p->loop_weight,
                                         p->h_shift, p->d_M, p->precision, all_roots, d_c, d_a, s);
    if (sq)
        return cos_connected_det_subsets(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->h_shift, p->d_M, p->precision,
                                         all_roots, d_c, d_a, s);
    if (loops)
        return cos_connected_sum_bipartite_subsets(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->n_mat,
                                                   p->loop_weight, p->h_shift, p->d_M, p->precision, all_roots, d_c,
                                                   d_a, s);
    return cos_connected_det_bipartite_subsets(p->n_cfg, p->n_max, p->d_order, p->d_moff, p->h_shift, p->d_M,
                                               p->precision, all_roots, d_c, d_a, s);
}
