// Sharded single registration: one rigid EM whose model points are split
// across ranks.  The E step's sums (Eq. 6, Eq. 9) and the Gauss-Newton sums of
// Eq. 17-18 are sums over model points, so each rank forms the normal
// equations of its own shard (fr_rigid_normal_equations on its GPU), the
// caller's collective adds the FR_NE_VALS values, and every rank solves the
// same 6 x 6 system and applies the same twist (Eq. 16, Eq. 18) -- the ranks
// hold identical poses without exchanging them.  The EM loop, the solve and
// the SE(3) update here are host code (a 6 x 6 system per iteration); the
// per-point work stays on the GPU.
#include "context.h"

#include <cmath>

using namespace fr;

namespace {

// Index of A[p][q] (p <= q) in the upper triangle stored row by row.
int tri(int p, int q) { return p * 6 - p * (p - 1) / 2 + (q - p); }

// delta zeta = -A^-1 b by LDL^T of the symmetric A; false if a pivot is at or
// below 1e-12 of the largest diagonal entry (or that entry is not positive).
bool solve6(const double *ne, double dz[6]) {
    double A[6][6];
    for (int p = 0; p < 6; ++p)
        for (int q = p; q < 6; ++q) A[p][q] = A[q][p] = ne[tri(p, q)];
    double md = 0.0;
    for (int p = 0; p < 6; ++p) md = std::fmax(md, A[p][p]);
    if (!(md > 0.0)) return false;
    const double floor_ = md * 1e-12;
    double L[6][6] = {}, Dg[6];
    for (int k = 0; k < 6; ++k) {
        double d = A[k][k];
        for (int j = 0; j < k; ++j) d -= L[k][j] * L[k][j] * Dg[j];
        if (!(d > floor_)) return false;
        Dg[k] = d;
        L[k][k] = 1.0;
        for (int i = k + 1; i < 6; ++i) {
            double v = A[i][k];
            for (int j = 0; j < k; ++j) v -= L[i][j] * L[k][j] * Dg[j];
            L[i][k] = v / d;
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {  // L y = -b
        double v = -ne[21 + i];
        for (int j = 0; j < i; ++j) v -= L[i][j] * y[j];
        y[i] = v;
    }
    for (int i = 0; i < 6; ++i) y[i] /= Dg[i];
    for (int i = 5; i >= 0; --i) {  // L^T dz = y
        double v = y[i];
        for (int j = i + 1; j < 6; ++j) v -= L[j][i] * dz[j];
        dz[i] = v;
    }
    return true;
}

// exp of the twist (omega; v) (Eq. 16): R = I + a W + b W^2, t = (I + b W +
// c W^2) v with a = sin(th)/th, b = (1 - cos th)/th^2, c = (th - sin th)/th^3
// (their Taylor series below th = 1e-4).
void se3_exp(const double z[6], double E[16]) {
    const double w[3] = {z[0], z[1], z[2]}, v[3] = {z[3], z[4], z[5]};
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = std::sqrt(th2);
    double a, b, c;
    if (th < 1e-4) {
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        c = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        a = std::sin(th) / th;
        b = (1.0 - std::cos(th)) / th2;
        c = (th - std::sin(th)) / (th2 * th);
    }
    const double W[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
    double W2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) W2[i][j] = W[i][0] * W[0][j] + W[i][1] * W[1][j] + W[i][2] * W[2][j];
    for (int i = 0; i < 3; ++i) {
        double t = 0.0;
        for (int j = 0; j < 3; ++j) {
            const double I = i == j ? 1.0 : 0.0;
            E[4 * i + j] = I + a * W[i][j] + b * W2[i][j];
            t += (I + b * W[i][j] + c * W2[i][j]) * v[j];
        }
        E[4 * i + 3] = t;
    }
    E[12] = E[13] = E[14] = 0.0;
    E[15] = 1.0;
}

fr_status as_status(int r) { return (r >= FR_OK && r <= FR_ENOTSUPPORTED) ? (fr_status)r : FR_ECUDA; }

}  // namespace

extern "C" FR_API fr_status fr_rigid_solve_update(const double ne[FR_NE_VALS], double T_inout[16],
                                                  double *twist_norm) {
    if (!ne || !T_inout) return FR_EINVAL;
    for (int i = 0; i < 27; ++i)
        if (!std::isfinite(ne[i])) return FR_EINVAL;
    double dz[6];
    if (!solve6(ne, dz)) return FR_EINVAL;
    double E[16], T[16];
    se3_exp(dz, E);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            T[4 * i + j] = E[4 * i] * T_inout[j] + E[4 * i + 1] * T_inout[4 + j] + E[4 * i + 2] * T_inout[8 + j] +
                           E[4 * i + 3] * T_inout[12 + j];
    for (int i = 0; i < 16; ++i) T_inout[i] = T[i];
    if (twist_norm) {
        double n2 = 0.0;
        for (int p = 0; p < 6; ++p) n2 += dz[p] * dz[p];
        *twist_norm = std::sqrt(n2);
    }
    return FR_OK;
}

extern "C" FR_API fr_status fr_em_sharded(fr_ne_fn ne_fn, void *ne_user, fr_allreduce_fn allreduce, void *ar_user,
                                          const fr_options *opt, double T_inout[16], fr_report *report) {
    if (!ne_fn || !opt || !T_inout) return FR_EINVAL;
    if (opt->iters < 0 || opt->iters > 100000) return FR_EINVAL;
    if (!(opt->sigma_start > 0.0f) || !(opt->sigma_end > 0.0f) || !std::isfinite(opt->sigma_start) ||
        !std::isfinite(opt->sigma_end))
        return FR_EINVAL;
    if (!(opt->w >= 0.0f && opt->w < 1.0f)) return FR_EINVAL;
    if (opt->update_sigma) return FR_ENOTSUPPORTED;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T_inout[i])) return FR_EINVAL;
    fr_report rep{};
    double ne[FR_NE_VALS];
    fr_status st = FR_OK;
    for (int k = 0; k < opt->iters; ++k) {
        const float sig = schedule_sigma(opt, k);
        int r = ne_fn(T_inout, sig, ne, ne_user);
        if (r != 0) {
            st = as_status(r);
            break;
        }
        if (allreduce) {
            r = allreduce(ne, FR_NE_VALS, ar_user);
            if (r != 0) {
                st = as_status(r);
                break;
            }
        }
        rep.iters_run = k + 1;
        rep.last_sum_w = ne[27];
        rep.last_cost = ne[28];
        rep.last_inliers = (int64_t)(ne[29] + 0.5);
        rep.last_sigma = sig;
        double tn = 0.0;
        if (fr_rigid_solve_update(ne, T_inout, &tn) != FR_OK) {
            rep.degenerate_iters += 1;
            continue;
        }
        rep.last_twist_norm = tn;
        if (opt->stop_twist > 0.0f && tn < (double)opt->stop_twist) break;
    }
    if (report) *report = rep;
    return st;
}

namespace {

struct GpuShard {
    fr_ctx *ctx;
    const float *X, *Y, *Yn;
    int64_t M, N, M_total;
    const fr_options *opt;
};

int gpu_shard_ne(const double T[16], float sigma, double *ne, void *user) {
    const GpuShard &g = *static_cast<const GpuShard *>(user);
    fr_options o = *g.opt;
    o.sigma_start = o.sigma_end = sigma;
    return fr_rigid_normal_equations(g.ctx, g.X, g.M, g.Y, g.Yn, g.N, &o, g.M_total, T, ne);
}

}  // namespace

extern "C" FR_API fr_status fr_register_rigid_sharded(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                                      const float *d_Yn, int64_t N, const fr_options *opt,
                                                      int64_t M_total, fr_allreduce_fn allreduce, void *ar_user,
                                                      double T_inout[16], fr_report *report) {
    fr::NvtxRange nvtx_("fr_register_rigid_sharded");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_options(ctx, opt));
    FR_TRY(validate_cloud(ctx, d_X, M, "d_X"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (opt->residual == FR_PT2PL) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn (normals, required for FR_PT2PL)"));
    if (M_total < M) return ctx->fail(FR_EINVAL, "M_total must be >= M");
    GpuShard g{ctx, d_X, d_Y, opt->residual == FR_PT2PL ? d_Yn : nullptr, M, N, M_total, opt};
    const fr_status st = fr_em_sharded(gpu_shard_ne, &g, allreduce, ar_user, opt, T_inout, report);
    if (st != FR_OK && ctx->err.empty()) ctx->fail(st, "sharded registration stopped (a callback failed)");
    return st;
}
