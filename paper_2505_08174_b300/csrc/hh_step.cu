// hh_step.cu -- the explicit Euler step of the filament suspension (the
// paper's application layer, Sections 2.5 and 4.3): bead forces from the chain
// potentials, the prediction U = M(X) F, and x <- x + dt U.
//
// Chains are `beads` consecutive rows of X.  With r_m = x_{m+1} - x_m,
// L_m = |r_m|, t_m = r_m / L_m along a chain, the energy is
//   E = sum_m (k/2)(L_m - l0)^2 + sum_m kappa (1 - t_m . t_{m+1}) - sum_i g . x_i
// (a harmonic bond spring as in Eq. 12 and a bending term written as the
// potential whose gradient it is).  Its gradient with respect to bond m is
//   dE/dr_m = k (L_m - l0) t_m
//             - kappa (t_{m+1} - (t_m . t_{m+1}) t_m) / L_m   (joint m, m+1)
//             - kappa (t_{m-1} - (t_{m-1} . t_m) t_m) / L_m   (joint m-1, m)
// and since r_{j-1} and r_j are the bonds that move with bead j,
//   F_j = -dE/dx_j = g - dE/dr_{j-1} + dE/dr_j.
// One thread per bead gathers the (at most four) bonds it needs, so each
// force is written once with no atomics; neighbouring threads read the same
// beads through L1.  FP64 throughout (a few hundred flops per bead).
#include "hh_internal.h"

namespace {

// dE/dr_m of bond m (beads m, m+1) of the chain starting at x; 0 <= m < beads-1.
// Returns false when a bond it reads has zero length.
__device__ bool bond_gradient(const double* __restrict__ x, int beads, int m, const FilamentArgs& a, double out[3])
{
    double t[3][3], L[3];
    bool has[3];
    bool ok = true;
    for (int q = 0; q < 3; ++q) {
        const int b = m - 1 + q;
        has[q] = b >= 0 && b + 1 < beads;
        if (!has[q]) continue;
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = x[3 * (b + 1) + d] - x[3 * b + d];
        L[q] = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        ok = ok && L[q] > 0.0;
        for (int d = 0; d < 3; ++d) t[q][d] = r[d] / L[q];
    }
    for (int d = 0; d < 3; ++d) out[d] = a.k * (L[1] - a.l0) * t[1][d];
    for (int q = 0; q < 3; q += 2) {
        if (!has[q]) continue;
        const double c = t[q][0] * t[1][0] + t[q][1] * t[1][1] + t[q][2] * t[1][2];
        for (int d = 0; d < 3; ++d) out[d] -= a.kappa * (t[q][d] - c * t[1][d]) / L[1];
    }
    return ok;
}

__global__ void k_filament_forces(const double* __restrict__ X, int64_t n_chains, int beads, FilamentArgs a,
                                  double* __restrict__ F, unsigned* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_chains * beads) return;
    const int64_t c = i / beads;
    const int j = (int)(i - c * beads);
    const double* x = X + 3 * c * beads;
    double f[3] = {a.g[0], a.g[1], a.g[2]};
    double gr[3];
    bool ok = true;
    if (j >= 1) {
        ok = bond_gradient(x, beads, j - 1, a, gr) && ok;
        for (int d = 0; d < 3; ++d) f[d] -= gr[d];
    }
    if (j + 1 < beads) {
        ok = bond_gradient(x, beads, j, a, gr) && ok;
        for (int d = 0; d < 3; ++d) f[d] += gr[d];
    }
    for (int d = 0; d < 3; ++d) ok = ok && isfinite(f[d]);
    if (!ok) atomicOr(status, (unsigned)HH_DEV_NUMERIC);
    for (int d = 0; d < 3; ++d) F[3 * i + d] = f[d];
}

__global__ void k_euler(double* __restrict__ X, const double* __restrict__ U, int64_t n3, double dt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) X[i] += dt * U[i];
}

}  // namespace

void filament_forces_launch(hh_ctx* ctx, const double* X, int64_t n_chains, int32_t beads, const FilamentArgs& a,
                            double* F, cudaStream_t s)
{
    const int64_t n = n_chains * beads;
    if (n == 0) return;
    k_filament_forces<<<(unsigned)ceil_div(n, (int64_t)256), 256, 0, s>>>(X, n_chains, beads, a, F, ctx->d_status);
    HH_CHECK_LAUNCH();
}

void euler_launch(double* X, const double* U, int64_t n3, double dt, cudaStream_t s)
{
    if (n3 == 0) return;
    k_euler<<<(unsigned)ceil_div(n3, (int64_t)256), 256, 0, s>>>(X, U, n3, dt);
    HH_CHECK_LAUNCH();
}
