// Discrete adjoint of the Euler and Navier-Stokes right-hand sides and of
// classical RK4.
//
// Not in the paper.  The transpose of R = -J^-1 [M3 D~ + (M1 - M3 M2) F~]
// (App. A) is applied by running the RHS steps backwards:
//   mu  = -J^-1 lambda                           (adj_scale)
//   g_D = M3^T mu,  g_F = (M1 - M3 M2)^T mu      (operator products)
//   per pair: a = |n|_L g_D,L - |n|_R g_D,R,  a_uL = (dF/duL)^T a,
//             a_uR = (dF/duR)^T a  with F the Rusanov flux (App. B), plus for
//             Navier-Stokes the LDG viscous part and tau penalty (Sec. 4.3):
//             a_qL, a_qR = (dF/dqL)^T a, (dF/dqR)^T a
//   per boundary point the ghost states' dependence on u_L (and q_L) is
//   included (App. C)
//   point-wise: a_u += (df/du)^T adj(J)^T g_F, and for Navier-Stokes
//             a_q = (df/dq)^T adj(J)^T g_F + M0^T a_qf, a_q~ = J^-1 a_q
//   Navier-Stokes gradient chain (Q~ = M6 C + (M4 - M6 M0) U):
//             a_C = M6^T a_q~, a_uf += (dC/duf)^T a_C (LDG common solution)
//   out = M0^T a_uf [+ (M4 - M6 M0)^T a_q~] + point-wise terms
// The local transposed Jacobians are written out analytically from the
// fluxes (Eq. eulerflux, idealgas, visflux), in plain (not perturbation)
// variables.  The Navier-Stokes adjoint recomputes U^(f), Q and Q^(f) at u
// with the forward kernels first.  The RK4 adjoint recomputes stage inputs
// from checkpoints.
#include <cmath>
#include <vector>

#include "../../include/fr.h"
#include "fr_dev.hpp"

namespace fr {

template <typename T, int D>
struct EulerAdj {
    static constexpr int NV = D + 2;

    // a += (d f_j,alpha / d u)^T G[j][alpha]
    __device__ static __forceinline__ void flux_vjp(const T* u, const T G[D][NV], T gamma, T* a) {
        const T gm1 = gamma - T(1), rho = u[0], rinv = T(1) / rho;
        T v[D], v2 = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * rinv; v2 += v[i] * v[i]; }
        const T p = gm1 * (u[D + 1] - T(0.5) * rho * v2);
        const T dp_drho = gm1 * T(0.5) * v2;
        T S = T(0), H = T(0), Gvv = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            S += G[j][1 + j];
            H += G[j][D + 1] * v[j];
#pragma unroll
            for (int i = 0; i < D; ++i) Gvv += G[j][1 + i] * v[i] * v[j];
        }
        const T EpR = (u[D + 1] + p) * rinv;
        a[0] += -Gvv + dp_drho * (S + H) - EpR * H;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            T acc = G[k][0] + G[k][D + 1] * EpR - gm1 * v[k] * (S + H);
#pragma unroll
            for (int j = 0; j < D; ++j) acc += (G[j][1 + k] + G[k][1 + j]) * v[j];
            a[1 + k] += acc;
        }
        a[D + 1] += gm1 * S + gamma * H;
    }

    __device__ static __forceinline__ void prim(const T* u, T gm1, T& rho, T* v, T& p) {
        rho = u[0];
        T rinv = T(1) / rho, v2 = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * rinv; v2 += v[i] * v[i]; }
        p = gm1 * (u[D + 1] - T(0.5) * rho * v2);
    }

    __device__ static __forceinline__ void normal_flux(const T* u, const T* n, T gm1, T* fn) {
        T rho, v[D], p;
        prim(u, gm1, rho, v, p);
        T vn = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) vn += n[i] * v[i];
        fn[0] = rho * vn;
#pragma unroll
        for (int i = 0; i < D; ++i) fn[1 + i] = u[1 + i] * vn + p * n[i];
        fn[D + 1] = (u[D + 1] + p) * vn;
    }

    // (dF/duL)^T a and (dF/duR)^T a for the Rusanov flux (App. B)
    __device__ static __forceinline__ void rusanov_vjp(const T* uL, const T* uR, const T* n, T gamma, const T* a,
                                                       T* aL, T* aR) {
        const T gm1 = gamma - T(1);
        T rL, vL[D], pL, rR, vR[D], pR;
        prim(uL, gm1, rL, vL, pL);
        prim(uR, gm1, rR, vR, pR);
        T q = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) q += n[i] * (vL[i] + vR[i]);
        const T cbar = sqrt(gamma * (pL + pR) / (rL + rR));
        const T s = cbar + T(0.5) * fabs(q);
        const T sgn = q >= T(0) ? T(1) : T(-1);
        T adu = T(0);
#pragma unroll
        for (int k = 0; k < NV; ++k) adu += a[k] * (uL[k] - uR[k]);
        // half of the normal-flux VJP on each side: G_j,alpha = n_j a_alpha / 2
        T G[D][NV];
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
            for (int k = 0; k < NV; ++k) G[j][k] = T(0.5) * n[j] * a[k];
#pragma unroll
        for (int k = 0; k < NV; ++k) { aL[k] = T(0.5) * s * a[k]; aR[k] = -T(0.5) * s * a[k]; }
        flux_vjp(uL, G, gamma, aL);
        flux_vjp(uR, G, gamma, aR);
        // d s / d u_X through cbar and |q|, times (a . (uL - uR)) / 2
        const T sum_r = rL + rR, sum_p = pL + pR;
        const T cfac = gamma / (T(2) * cbar);
        const T h = T(0.5) * adu;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const T* v = side == 0 ? vL : vR;
            const T rho = side == 0 ? rL : rR;
            T* out = side == 0 ? aL : aR;
            T v2 = T(0), vn = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) { v2 += v[i] * v[i]; vn += n[i] * v[i]; }
            // dp/drho = gm1 |v|^2 / 2, dp/dm_k = -gm1 v_k, dp/dE = gm1
            out[0] += h * (cfac * (gm1 * T(0.5) * v2 / sum_r - sum_p / (sum_r * sum_r)) + T(0.5) * sgn * (-vn / rho));
#pragma unroll
            for (int k = 0; k < D; ++k) out[1 + k] += h * (cfac * (-gm1 * v[k]) / sum_r + T(0.5) * sgn * n[k] / rho);
            out[D + 1] += h * cfac * gm1 / sum_r;
        }
    }

    // inviscid ghost state (App. C), plain variables, and the transpose of
    // its Jacobian applied to b (added to c)
    __device__ static __forceinline__ void ghost(int bctype, const T* uL, const DevParams& P, T* g) {
        const T gamma = T(P.gamma), gm1 = gamma - T(1);
        if (bctype == 0) {
            T rho = T(P.bc_rho), ke = T(0);
            g[0] = rho;
#pragma unroll
            for (int i = 0; i < D; ++i) { g[1 + i] = rho * T(P.bc_v[i]); ke += T(P.bc_v[i]) * T(P.bc_v[i]); }
            g[D + 1] = T(P.bc_p) / gm1 + T(0.5) * rho * ke;
        } else if (bctype == 1) {
            T ke = T(0);
            g[0] = uL[0];
#pragma unroll
            for (int i = 0; i < D; ++i) { g[1 + i] = uL[1 + i]; ke += uL[1 + i] * uL[1 + i]; }
            g[D + 1] = T(P.outflow_p) / gm1 + T(0.5) * ke / uL[0];
        } else {
            const double* wv = bctype == 3 ? P.wall2_v : P.wall_v;
            const T rho = uL[0], rinv = T(1) / rho;
            T k1 = T(0);
            g[0] = rho;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T w = T(2) * T(wv[i]) - uL[1 + i] * rinv;
                g[1 + i] = rho * w;
                k1 += w * w;
            }
            g[D + 1] = rho * (T(P.wall_cpTw) / gamma + T(0.5) * k1);
        }
    }

    __device__ static __forceinline__ void ghost_vjp(int bctype, const T* uL, const DevParams& P, const T* b, T* c) {
        if (bctype == 0) return;
        const T rho = uL[0], rinv = T(1) / rho;
        T v[D], v2 = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) { v[i] = uL[1 + i] * rinv; v2 += v[i] * v[i]; }
        if (bctype == 1) {
            c[0] += b[0] - T(0.5) * v2 * b[D + 1];
#pragma unroll
            for (int k = 0; k < D; ++k) c[1 + k] += b[1 + k] + v[k] * b[D + 1];
            return;
        }
        const double* vwall = bctype == 3 ? P.wall2_v : P.wall_v;
        T w[D], w2 = T(0), wv = T(0), bm = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            w[i] = T(2) * T(vwall[i]) - v[i];
            w2 += w[i] * w[i];
            wv += w[i] * v[i];
            bm += T(2) * T(vwall[i]) * b[1 + i];
        }
        c[0] += b[0] + bm + (T(P.wall_cpTw) / T(P.gamma) + T(0.5) * w2 + wv) * b[D + 1];
#pragma unroll
        for (int k = 0; k < D; ++k) c[1 + k] += -b[1 + k] - w[k] * b[D + 1];
    }
};

template <typename T, int D>
struct NsAdj {
    static constexpr int NV = D + 2;

    // Viscous flux (Eq. visflux, constant mu, kappa = mu gamma / (Pr (gamma-1))
    // multiplying grad(p/rho)) in plain variables, differentiated in reverse:
    // au += (d f_vis / du)^T W and aq += (d f_vis / dq)^T W, where W[i][a]
    // weights f_vis[i][a].
    __device__ static __forceinline__ void vis_vjp(const T* u, const T q[D][NV], const T W[D][NV], T gm1, T mu,
                                                   T kappa, T* au, T aq[D][NV]) {
        const T rho = u[0], rinv = T(1) / rho;
        T v[D], v2 = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * rinv; v2 += v[i] * v[i]; }
        const T p = gm1 * (u[D + 1] - T(0.5) * rho * v2), pr = p * rinv;
        // forward: dv[i][j] = d v_i / d x_j, dpr[j] = d (p/rho) / d x_j, stress tau
        T dv[D][D], dpr[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T drho = q[j][0];
            T vdm = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) { dv[i][j] = (q[j][1 + i] - v[i] * drho) * rinv; vdm += v[i] * q[j][1 + i]; }
            const T dp = gm1 * (q[j][D + 1] - vdm + T(0.5) * v2 * drho);
            dpr[j] = (dp - pr * drho) * rinv;
        }
        T div = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) div += dv[i][i];
        // reverse: adjoints of tau (Wt), of v (av), of grad(p/rho) (Wdpr)
        T Wt[D][D], av[D], trW = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int j = 0; j < D; ++j) Wt[i][j] = W[i][1 + j] + v[i] * W[j][D + 1];
            trW += Wt[i][i];
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const T tji = mu * (dv[i][j] + dv[j][i]) - (i == j ? T(2) / T(3) * mu * div : T(0));
                acc += W[i][D + 1] * tji;
            }
            av[j] = acc;
        }
        T arinv = T(0), apr = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            // dv[k][j] = (q[j][1+k] - v_k q[j][0]) / rho
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T w = mu * (Wt[j][k] + Wt[k][j]) - (k == j ? T(2) / T(3) * mu * trW : T(0));   // adjoint of dv[k][j]
                aq[j][1 + k] += w * rinv;
                aq[j][0] -= w * v[k] * rinv;
                av[k] -= w * q[j][0] * rinv;
                arinv += w * dv[k][j] * rho;
            }
            // dpr[j] = (dp_j - (p/rho) q[j][0]) / rho,
            // dp_j = gm1 (q[j][E] - v . q[j][m] + |v|^2 q[j][0] / 2)
            const T wpr = kappa * W[j][D + 1];
            const T wdp = wpr * rinv;
            aq[j][0] += -wpr * pr * rinv + gm1 * wdp * T(0.5) * v2;
            apr -= wpr * q[j][0] * rinv;
            arinv += wpr * dpr[j] * rho;
            aq[j][D + 1] += gm1 * wdp;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                aq[j][1 + k] -= gm1 * wdp * v[k];
                av[k] += gm1 * wdp * (v[k] * q[j][0] - q[j][1 + k]);
            }
        }
        // p/rho = p * (1/rho)
        const T ap = apr * rinv;
        arinv += apr * p;
        // to conserved variables: p = gm1 (E - |m|^2 / (2 rho)), v = m / rho, 1/rho
        T avv = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            au[1 + k] += -gm1 * v[k] * ap + av[k] * rinv;
            avv += av[k] * v[k];
        }
        au[D + 1] += gm1 * ap;
        au[0] += gm1 * T(0.5) * v2 * ap - avv * rinv - arinv * rinv * rinv;
    }

    // LDG ghost state (App. C) in plain variables: the inviscid ghost for
    // free-stream and outflow faces; at isothermal walls the wall velocity
    // and temperature with the interior density
    __device__ static __forceinline__ void ldg_ghost(int bctype, const T* uL, const DevParams& P, T* g) {
        if (bctype <= 1) { EulerAdj<T, D>::ghost(bctype, uL, P, g); return; }
        const double* wv = bctype == 3 ? P.wall2_v : P.wall_v;
        const T rho = uL[0];
        T k2 = T(0);
        g[0] = rho;
#pragma unroll
        for (int i = 0; i < D; ++i) { g[1 + i] = rho * T(wv[i]); k2 += T(wv[i]) * T(wv[i]); }
        g[D + 1] = rho * (T(P.wall_cpTw) / T(P.gamma) + T(0.5) * k2);
    }

    // c += (d ldg_ghost / d uL)^T b
    __device__ static __forceinline__ void ldg_ghost_vjp(int bctype, const T* uL, const DevParams& P, const T* b,
                                                         T* c) {
        if (bctype <= 1) { EulerAdj<T, D>::ghost_vjp(bctype, uL, P, b, c); return; }
        const double* wv = bctype == 3 ? P.wall2_v : P.wall_v;
        T k2 = T(0), bm = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) { k2 += T(wv[i]) * T(wv[i]); bm += T(wv[i]) * b[1 + i]; }
        c[0] += b[0] + bm + (T(P.wall_cpTw) / T(P.gamma) + T(0.5) * k2) * b[D + 1];
    }

    // weights of the viscous part of the common flux on one side:
    // W[i][a] = -w n_i a_a (F contains -n . w f_vis)
    __device__ static __forceinline__ void side_weights(const T* n, const T* a, T w, T W[D][NV]) {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < NV; ++k) W[i][k] = -w * n[i] * a[k];
    }
};

// mu = -lambda / J
template <typename T>
__global__ void adj_scale_kernel(int nupts, int nvars, int64_t nelem, int64_t ld, const T* __restrict__ lam,
                                 const T* __restrict__ rcp, T* __restrict__ mu) {
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = blockIdx.y;
    if (n >= nelem) return;
    T r = rcp[(int64_t)s * ld + n];
    for (int a = 0; a < nvars; ++a) {
        int64_t i = ((int64_t)s * nvars + a) * ld + n;
        mu[i] = -lam[i] * r;
    }
}

// pairs: a = |n|_L g_D,L - |n|_R g_D,R; write (dF/duL)^T a, (dF/duR)^T a in place of g_D
template <typename T, int D>
__global__ void adj_pair_kernel(int64_t npairs, const uint32_t* __restrict__ offL, const uint32_t* __restrict__ offR,
                                const T* __restrict__ ufL, const T* __restrict__ ufR, T* gL, T* gR, int64_t ldL,
                                int64_t ldR, const T* __restrict__ nrm, const T* __restrict__ magL,
                                const T* __restrict__ magR, T gamma) {
    constexpr int NV = D + 2;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    int64_t oL = offL[k], oR = offR[k];
    T uL[NV], uR[NV], a[NV], n[D], aL[NV], aR[NV];
    const T mL = magL[k], mR = magR[k];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        uL[q] = ufL[oL + q * ldL];
        uR[q] = ufR[oR + q * ldR];
        a[q] = mL * gL[oL + q * ldL] - mR * gR[oR + q * ldR];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) n[i] = nrm[i * npairs + k];
    EulerAdj<T, D>::rusanov_vjp(uL, uR, n, gamma, a, aL, aR);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        gL[oL + q * ldL] = aL[q];
        gR[oR + q * ldR] = aR[q];
    }
}

template <typename T, int D>
__global__ void adj_bc_kernel(int64_t nb, int bctype, const uint32_t* __restrict__ off, const T* __restrict__ uf,
                              T* g, int64_t ld, const T* __restrict__ nrm, const T* __restrict__ mag, DevParams P) {
    constexpr int NV = D + 2;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    int64_t o = off[k];
    T uL[NV], gs[NV], a[NV], n[D], aL[NV], aR[NV];
    const T m = mag[k];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        uL[q] = uf[o + q * ld];
        a[q] = m * g[o + q * ld];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) n[i] = nrm[i * nb + k];
    EulerAdj<T, D>::ghost(bctype, uL, P, gs);
    EulerAdj<T, D>::rusanov_vjp(uL, gs, n, T(P.gamma), a, aL, aR);
    EulerAdj<T, D>::ghost_vjp(bctype, uL, P, aR, aL);
#pragma unroll
    for (int q = 0; q < NV; ++q) g[o + q * ld] = aL[q];
}

// out += (df/du)^T adj(J)^T g_F at solution points
template <typename T, int D>
__global__ void adj_flux_kernel(int nupts, int64_t nelem, int64_t ld, const T* __restrict__ U,
                                const T* __restrict__ gF, const T* __restrict__ smat, T* out, T gamma) {
    constexpr int NV = D + 2;
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = blockIdx.y;
    if (n >= nelem) return;
    T u[NV], G[D][NV], adj[D][D], a[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        u[q] = U[((int64_t)s * NV + q) * ld + n];
        a[q] = T(0);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) adj[i][j] = smat[((int64_t)(i * D + j) * nupts + s) * ld + n];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) acc += adj[i][j] * gF[((int64_t)(i * nupts + s) * NV + q) * ld + n];
            G[j][q] = acc;
        }
    EulerAdj<T, D>::flux_vjp(u, G, gamma, a);
#pragma unroll
    for (int q = 0; q < NV; ++q) out[((int64_t)s * NV + q) * ld + n] += a[q];
}

// Navier-Stokes pairs: the common flux F = Rusanov - n.{(1/2+b) fv_L +
// (1/2-b) fv_R} + tau (u_L - u_R) transposed; a_u in place of g_D, a_q in
// place of Q^(f)
template <typename T, int D>
__global__ void ns_adj_pair_kernel(int64_t npairs, const uint32_t* __restrict__ offL,
                                   const uint32_t* __restrict__ offR, const T* __restrict__ ufL,
                                   const T* __restrict__ ufR, T* gL, T* gR, T* qfL, T* qfR, int64_t ldL, int64_t ldR,
                                   int64_t qsL, int64_t qsR, const T* __restrict__ nrm, const T* __restrict__ magL,
                                   const T* __restrict__ magR, DevParams P) {
    constexpr int NV = D + 2;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    const int64_t oL = offL[k], oR = offR[k];
    const T gamma = T(P.gamma), gm1 = gamma - T(1), mu = T(P.mu), tau = T(P.tau), beta = T(P.beta);
    const T kappa = T(P.mu * P.gamma / (P.prandtl * (P.gamma - 1.0)));
    T uL[NV], uR[NV], a[NV], n[D], aL[NV], aR[NV];
    const T mL = magL[k], mR = magR[k];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        uL[q] = ufL[oL + q * ldL];
        uR[q] = ufR[oR + q * ldR];
        a[q] = mL * gL[oL + q * ldL] - mR * gR[oR + q * ldR];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) n[i] = nrm[i * npairs + k];
    EulerAdj<T, D>::rusanov_vjp(uL, uR, n, gamma, a, aL, aR);
#pragma unroll
    for (int q = 0; q < NV; ++q) { aL[q] += tau * a[q]; aR[q] -= tau * a[q]; }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const T* u = side == 0 ? uL : uR;
        T* au = side == 0 ? aL : aR;
        T* qf = side == 0 ? qfL : qfR;
        const int64_t o = side == 0 ? oL : oR, ld = side == 0 ? ldL : ldR, qs = side == 0 ? qsL : qsR;
        T q[D][NV], W[D][NV], aq[D][NV];
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
            for (int v = 0; v < NV; ++v) { q[j][v] = qf[j * qs + o + v * ld]; aq[j][v] = T(0); }
        NsAdj<T, D>::side_weights(n, a, side == 0 ? T(0.5) + beta : T(0.5) - beta, W);
        NsAdj<T, D>::vis_vjp(u, q, W, gm1, mu, kappa, au, aq);
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[j * qs + o + v * ld] = aq[j][v];
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        gL[oL + q * ldL] = aL[q];
        gR[oR + q * ldR] = aR[q];
    }
}

// Navier-Stokes boundary points: Rusanov with the inviscid ghost, the LDG
// viscous part and tau penalty with the LDG ghost and ghost gradient (q_L at
// walls, zero otherwise), all transposed onto u_L and q_L
template <typename T, int D>
__global__ void ns_adj_bc_kernel(int64_t nb, int bctype, const uint32_t* __restrict__ off, const T* __restrict__ uf,
                                 T* g, T* qf, int64_t ld, int64_t qs, const T* __restrict__ nrm,
                                 const T* __restrict__ mag, DevParams P) {
    constexpr int NV = D + 2;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int64_t o = off[k];
    const T gamma = T(P.gamma), gm1 = gamma - T(1), mu = T(P.mu), tau = T(P.tau), beta = T(P.beta);
    const T kappa = T(P.mu * P.gamma / (P.prandtl * (P.gamma - 1.0)));
    T uL[NV], gs[NV], gl[NV], a[NV], n[D], aL[NV], aR[NV], agl[NV];
    const T m = mag[k];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        uL[q] = uf[o + q * ld];
        a[q] = m * g[o + q * ld];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) n[i] = nrm[i * nb + k];
    EulerAdj<T, D>::ghost(bctype, uL, P, gs);
    EulerAdj<T, D>::rusanov_vjp(uL, gs, n, gamma, a, aL, aR);
    EulerAdj<T, D>::ghost_vjp(bctype, uL, P, aR, aL);
    NsAdj<T, D>::ldg_ghost(bctype, uL, P, gl);
#pragma unroll
    for (int q = 0; q < NV; ++q) { aL[q] += tau * a[q]; agl[q] = -tau * a[q]; }
    const bool wall = bctype >= 2;
    T q[D][NV], W[D][NV], aq[D][NV];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) { q[j][v] = qf[j * qs + o + v * ld]; aq[j][v] = T(0); }
    NsAdj<T, D>::side_weights(n, a, T(0.5) + beta, W);
    NsAdj<T, D>::vis_vjp(uL, q, W, gm1, mu, kappa, aL, aq);
    {
        // ghost side: gradient q_L at walls (its adjoint joins a_q), zero otherwise
        T qg[D][NV], aqg[D][NV];
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
            for (int v = 0; v < NV; ++v) { qg[j][v] = wall ? q[j][v] : T(0); aqg[j][v] = T(0); }
        NsAdj<T, D>::side_weights(n, a, T(0.5) - beta, W);
        NsAdj<T, D>::vis_vjp(gl, qg, W, gm1, mu, kappa, agl, aqg);
        if (wall)
#pragma unroll
            for (int j = 0; j < D; ++j)
#pragma unroll
                for (int v = 0; v < NV; ++v) aq[j][v] += aqg[j][v];
    }
    NsAdj<T, D>::ldg_ghost_vjp(bctype, uL, P, agl, aL);
#pragma unroll
    for (int q2 = 0; q2 < NV; ++q2) g[o + q2 * ld] = aL[q2];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) qf[j * qs + o + v * ld] = aq[j][v];
}

// Navier-Stokes solution points: G = adj(J)^T g_F;  a_u = (df_inv/du)^T G -
// (df_vis/du)^T G into au;  a_q = -(df_vis/dq)^T G + X (X = M0^T a_qf);
// a_q~ = adj(J) a_q / det J in place of Q
template <typename T, int D>
__global__ void ns_adj_point_kernel(int nupts, int64_t nelem, int64_t ld, const T* __restrict__ U, T* Q,
                                    const T* __restrict__ gF, const T* __restrict__ X, const T* __restrict__ smat,
                                    const T* __restrict__ rcp, T* __restrict__ au, DevParams P) {
    constexpr int NV = D + 2;
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = blockIdx.y;
    if (n >= nelem) return;
    const T gamma = T(P.gamma), gm1 = gamma - T(1), mu = T(P.mu);
    const T kappa = T(P.mu * P.gamma / (P.prandtl * (P.gamma - 1.0)));
    T u[NV], G[D][NV], adj[D][D], a[NV], q[D][NV], aq[D][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        u[v] = U[((int64_t)s * NV + v) * ld + n];
        a[v] = T(0);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) adj[i][j] = smat[((int64_t)(i * D + j) * nupts + s) * ld + n];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) acc += adj[i][j] * gF[((int64_t)(i * nupts + s) * NV + v) * ld + n];
            G[j][v] = acc;
            q[j][v] = Q[((int64_t)(j * nupts + s) * NV + v) * ld + n];
            aq[j][v] = X[((int64_t)(j * nupts + s) * NV + v) * ld + n];
        }
    EulerAdj<T, D>::flux_vjp(u, G, gamma, a);
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) G[j][v] = -G[j][v];
    NsAdj<T, D>::vis_vjp(u, q, G, gm1, mu, kappa, a, aq);
    const T r = rcp[(int64_t)s * ld + n];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < D; ++j) acc += adj[i][j] * aq[j][v];
            Q[((int64_t)(i * nupts + s) * NV + v) * ld + n] = acc * r;
        }
#pragma unroll
    for (int v = 0; v < NV; ++v) au[((int64_t)s * NV + v) * ld + n] = a[v];
}

// LDG common solution transposed (Sec. 4.3): both sides of a pair hold
// C = (1/2-b) u_L + (1/2+b) u_R, so a = a_C,L + a_C,R feeds both sides
template <typename T, int D>
__global__ void ns_adj_csol_kernel(int64_t npairs, const uint32_t* __restrict__ offL,
                                   const uint32_t* __restrict__ offR, const T* __restrict__ cL,
                                   const T* __restrict__ cR, T* aL, T* aR, int64_t ldL, int64_t ldR, T beta) {
    constexpr int NV = D + 2;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    const int64_t oL = offL[k], oR = offR[k];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const T ac = cL[oL + v * ldL] + cR[oR + v * ldR];
        aL[oL + v * ldL] += (T(0.5) - beta) * ac;
        aR[oR + v * ldR] += (T(0.5) + beta) * ac;
    }
}

// boundary: C = (1/2-b) u_L + (1/2+b) B_ldg(u_L)
template <typename T, int D>
__global__ void ns_adj_csol_bc_kernel(int64_t nb, int bctype, const uint32_t* __restrict__ off,
                                      const T* __restrict__ uf, const T* __restrict__ c, T* a, int64_t ld,
                                      DevParams P) {
    constexpr int NV = D + 2;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int64_t o = off[k];
    const T beta = T(P.beta);
    T uL[NV], gb[NV], res[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        uL[v] = uf[o + v * ld];
        const T cv = c[o + v * ld];
        res[v] = (T(0.5) - beta) * cv;
        gb[v] = (T(0.5) + beta) * cv;
    }
    NsAdj<T, D>::ldg_ghost_vjp(bctype, uL, P, gb, res);
#pragma unroll
    for (int v = 0; v < NV; ++v) a[o + v * ld] += res[v];
}

template <typename T>
__global__ void lincomb_kernel(int64_t n, T* out, T a, const T* x, T b,
                               const T* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = a * x[i] + (y ? b * y[i] : T(0));
}

static inline unsigned lgrid(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename T, int D>
static cudaError_t adjoint_impl(DevCtx& c, void* const* u, void* const* lam, void* const* out, cudaStream_t st) {
    const T gamma = T(c.prm.gamma);
    for (size_t b = 0; b < c.blocks.size(); ++b) {
        DevBlock& B = c.blocks[b];
        dim3 g((unsigned)((B.nelem + 127) / 128), (unsigned)B.nupts);
        adj_scale_kernel<T><<<g, 128, 0, st>>>(B.nupts, B.nvars, B.nelem, B.ld, (const T*)lam[b],
                                               (const T*)B.rcpdjac, (T*)B.adj_mu);
        cudaError_t e;
        if ((e = adjoint_gemm(c, 0, (int)b, u[b], B.adj_uf, st)) != cudaSuccess) return e;     // u^(f) = M0 u
        if ((e = adjoint_gemm(c, 1, (int)b, B.adj_mu, B.Uf, st)) != cudaSuccess) return e;     // g_D
        if ((e = adjoint_gemm(c, 2, (int)b, B.adj_mu, B.Q, st)) != cudaSuccess) return e;      // g_F
    }
    for (auto& g : c.pgroups) {
        if (!g.n) continue;
        DevBlock &L = c.blocks[g.bL], &R = c.blocks[g.bR];
        adj_pair_kernel<T, D><<<lgrid(g.n, 128), 128, 0, st>>>(g.n, g.offL, g.offR, (const T*)L.adj_uf,
                                                               (const T*)R.adj_uf, (T*)L.Uf, (T*)R.Uf, L.ld, R.ld,
                                                               (const T*)g.nrm, (const T*)g.magL, (const T*)g.magR,
                                                               gamma);
    }
    for (auto& g : c.bgroups) {
        if (!g.n) continue;
        DevBlock& B = c.blocks[g.b];
        adj_bc_kernel<T, D><<<lgrid(g.n, 128), 128, 0, st>>>(g.n, g.bctype, g.off, (const T*)B.adj_uf, (T*)B.Uf,
                                                             B.ld, (const T*)g.nrm, (const T*)g.mag, c.prm);
    }
    for (size_t b = 0; b < c.blocks.size(); ++b) {
        DevBlock& B = c.blocks[b];
        cudaError_t e;
        if ((e = adjoint_gemm(c, 3, (int)b, B.Uf, out[b], st)) != cudaSuccess) return e;       // M0^T a_uf
        dim3 g((unsigned)((B.nelem + 127) / 128), (unsigned)B.nupts);
        adj_flux_kernel<T, D><<<g, 128, 0, st>>>(B.nupts, B.nelem, B.ld, (const T*)u[b], (const T*)B.Q,
                                                 (const T*)B.smat, (T*)out[b], gamma);
    }
    return cudaGetLastError();
}

template <typename T, int D>
static cudaError_t ns_adjoint_impl(DevCtx& c, void* const* u, void* const* lam, void* const* out, cudaStream_t st) {
    constexpr int NV = D + 2;
    cudaError_t e;
    // forward values at u: plain U^(f) (adj_uf); Q (B.Q) and Q^(f) (B.Qf) by
    // the forward kernels (their U^(f) in B.Uf is not used)
    for (size_t b = 0; b < c.blocks.size(); ++b)
        if ((e = adjoint_gemm(c, 0, (int)b, u[b], c.blocks[b].adj_uf, st)) != cudaSuccess) return e;
    if ((e = launch_rhs_phases(c, u, nullptr, PH_A | PH_B1 | PH_B2, st)) != cudaSuccess) return e;
    for (size_t b = 0; b < c.blocks.size(); ++b) {
        DevBlock& B = c.blocks[b];
        dim3 g((unsigned)((B.nelem + 127) / 128), (unsigned)B.nupts);
        adj_scale_kernel<T><<<g, 128, 0, st>>>(B.nupts, B.nvars, B.nelem, B.ld, (const T*)lam[b],
                                               (const T*)B.rcpdjac, (T*)B.adj_mu);
        if ((e = adjoint_gemm(c, 1, (int)b, B.adj_mu, B.Uf, st)) != cudaSuccess) return e;     // g_D
        if ((e = adjoint_gemm(c, 2, (int)b, B.adj_mu, B.adj_g, st)) != cudaSuccess) return e;  // g_F
    }
    for (auto& g : c.pgroups) {
        if (!g.n) continue;
        DevBlock &L = c.blocks[g.bL], &R = c.blocks[g.bR];
        const int64_t qsL = (int64_t)L.nfpts * NV * L.ld, qsR = (int64_t)R.nfpts * NV * R.ld;
        ns_adj_pair_kernel<T, D><<<lgrid(g.n, 128), 128, 0, st>>>(
            g.n, g.offL, g.offR, (const T*)L.adj_uf, (const T*)R.adj_uf, (T*)L.Uf, (T*)R.Uf, (T*)L.Qf, (T*)R.Qf,
            L.ld, R.ld, qsL, qsR, (const T*)g.nrm, (const T*)g.magL, (const T*)g.magR, c.prm);
    }
    for (auto& g : c.bgroups) {
        if (!g.n) continue;
        DevBlock& B = c.blocks[g.b];
        ns_adj_bc_kernel<T, D><<<lgrid(g.n, 128), 128, 0, st>>>(g.n, g.bctype, g.off, (const T*)B.adj_uf, (T*)B.Uf,
                                                                (T*)B.Qf, B.ld, (int64_t)B.nfpts * NV * B.ld,
                                                                (const T*)g.nrm, (const T*)g.mag, c.prm);
    }
    for (size_t b = 0; b < c.blocks.size(); ++b) {
        DevBlock& B = c.blocks[b];
        const int64_t N = (int64_t)NV * B.ld;
        for (int j = 0; j < D; ++j)   // M0^T per direction of the flux-point gradient adjoint
            if ((e = adjoint_gemm(c, 3, (int)b, (const T*)B.Qf + (int64_t)j * B.nfpts * N,
                                  (T*)B.adj_x + (int64_t)j * B.nupts * N, st)) != cudaSuccess)
                return e;
        dim3 g((unsigned)((B.nelem + 127) / 128), (unsigned)B.nupts);
        ns_adj_point_kernel<T, D><<<g, 128, 0, st>>>(B.nupts, B.nelem, B.ld, (const T*)u[b], (T*)B.Q,
                                                     (const T*)B.adj_g, (const T*)B.adj_x, (const T*)B.smat,
                                                     (const T*)B.rcpdjac, (T*)B.adj_mu, c.prm);
        if ((e = adjoint_gemm(c, 4, (int)b, B.Q, B.Qf, st)) != cudaSuccess) return e;          // a_C = M6^T a_q~
    }
    for (auto& g : c.pgroups) {
        if (!g.n) continue;
        DevBlock &L = c.blocks[g.bL], &R = c.blocks[g.bR];
        ns_adj_csol_kernel<T, D><<<lgrid(g.n, 128), 128, 0, st>>>(g.n, g.offL, g.offR, (const T*)L.Qf,
                                                                  (const T*)R.Qf, (T*)L.Uf, (T*)R.Uf, L.ld, R.ld,
                                                                  T(c.prm.beta));
    }
    for (auto& g : c.bgroups) {
        if (!g.n) continue;
        DevBlock& B = c.blocks[g.b];
        ns_adj_csol_bc_kernel<T, D><<<lgrid(g.n, 128), 128, 0, st>>>(g.n, g.bctype, g.off, (const T*)B.adj_uf,
                                                                     (const T*)B.Qf, (T*)B.Uf, B.ld, c.prm);
    }
    for (size_t b = 0; b < c.blocks.size(); ++b) {
        DevBlock& B = c.blocks[b];
        // out = M0^T a_uf + (M4 - M6 M0)^T a_q~, then the point-wise terms
        if ((e = adjoint_gemm(c, 5, (int)b, B.Uf, out[b], st, B.Q)) != cudaSuccess) return e;
        const int64_t n = (int64_t)B.nupts * NV * B.ld;
        lincomb_kernel<T><<<lgrid(n, 256), 256, 0, st>>>(n, (T*)out[b], T(1), (const T*)out[b], T(1),
                                                         (const T*)B.adj_mu);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_rhs(DevCtx& c, void* const* u, void* const* lam, void* const* out, cudaStream_t st) {
    if (c.system == 1) {
        if (c.precision == 0) return c.ndims == 2 ? ns_adjoint_impl<double, 2>(c, u, lam, out, st)
                                                  : ns_adjoint_impl<double, 3>(c, u, lam, out, st);
        return c.ndims == 2 ? ns_adjoint_impl<float, 2>(c, u, lam, out, st)
                            : ns_adjoint_impl<float, 3>(c, u, lam, out, st);
    }
    if (c.precision == 0) return c.ndims == 2 ? adjoint_impl<double, 2>(c, u, lam, out, st)
                                              : adjoint_impl<double, 3>(c, u, lam, out, st);
    return c.ndims == 2 ? adjoint_impl<float, 2>(c, u, lam, out, st) : adjoint_impl<float, 3>(c, u, lam, out, st);
}

// ---------------------------------------------------------------- RK4 adjoint
template <typename T>
static cudaError_t rk4_adjoint_impl(DevCtx& c, void* const* u0, void* const* lam, double dt, int nsteps, int every,
                                    const std::vector<std::vector<void*>>& ck, const std::vector<std::vector<void*>>& blk,
                                    const std::vector<std::vector<void*>>& tmp, cudaStream_t st) {
    const size_t nb = c.blocks.size();
    auto nval = [&](size_t b) { return (int64_t)c.blocks[b].nupts * c.blocks[b].nvars * c.blocks[b].ld; };
    auto copy = [&](const std::vector<void*>& dst, void* const* src) {
        for (size_t b = 0; b < nb; ++b)
            cudaMemcpyAsync(dst[b], src[b], nval(b) * sizeof(T), cudaMemcpyDeviceToDevice, st);
    };
    auto comb = [&](const std::vector<void*>& out, double a, void* const* x, double bb, void* const* y) {
        for (size_t b = 0; b < nb; ++b)
            lincomb_kernel<T><<<lgrid(nval(b), 256), 256, 0, st>>>(nval(b), (T*)out[b], T(a), (const T*)x[b], T(bb),
                                                                   y ? (const T*)y[b] : nullptr);
    };
    // tmp slots: 0..3 stage inputs y1..y4, 4 k, 5 t, 6 w, 7 sum
    const auto &y1 = tmp[0], &y2 = tmp[1], &y3 = tmp[2], &y4 = tmp[3], &k = tmp[4], &t = tmp[5], &w = tmp[6],
               &sum = tmp[7];
    cudaError_t e;
    // forward sweep: checkpoint i holds u_{i * every}
    copy(ck[0], u0);
    for (size_t i = 1; i < ck.size(); ++i) {
        copy(ck[i], ck[i - 1].data());
        if ((e = launch_rk4(c, (void* const*)ck[i].data(), dt, every, st)) != cudaSuccess) return e;
    }
    // backward sweep, one checkpoint block at a time
    for (int blk0 = ((nsteps - 1) / every) * every; blk0 >= 0; blk0 -= every) {
        const int len = std::min(every, nsteps - blk0);
        copy(blk[0], ck[blk0 / every].data());
        for (int j = 1; j < len; ++j) {
            copy(blk[j], blk[j - 1].data());
            if ((e = launch_rk4(c, (void* const*)blk[j].data(), dt, 1, st)) != cudaSuccess) return e;
        }
        for (int j = len - 1; j >= 0; --j) {
            void* const* un = blk[j].data();
            // stage inputs
            copy(y1, un);
            if ((e = launch_rhs(c, y1.data(), k.data(), st)) != cudaSuccess) return e;
            comb(y2, 1.0, un, 0.5 * dt, k.data());
            if ((e = launch_rhs(c, y2.data(), k.data(), st)) != cudaSuccess) return e;
            comb(y3, 1.0, un, 0.5 * dt, k.data());
            if ((e = launch_rhs(c, y3.data(), k.data(), st)) != cudaSuccess) return e;
            comb(y4, 1.0, un, dt, k.data());
            // adjoint of the step
            comb(t, dt / 6.0, lam, 0.0, nullptr);
            if ((e = launch_adjoint_rhs(c, y4.data(), t.data(), w.data(), st)) != cudaSuccess) return e;
            copy(sum, w.data());
            comb(t, dt / 3.0, lam, dt, w.data());
            if ((e = launch_adjoint_rhs(c, y3.data(), t.data(), w.data(), st)) != cudaSuccess) return e;
            comb(sum, 1.0, sum.data(), 1.0, w.data());
            comb(t, dt / 3.0, lam, 0.5 * dt, w.data());
            if ((e = launch_adjoint_rhs(c, y2.data(), t.data(), w.data(), st)) != cudaSuccess) return e;
            comb(sum, 1.0, sum.data(), 1.0, w.data());
            comb(t, dt / 6.0, lam, 0.5 * dt, w.data());
            if ((e = launch_adjoint_rhs(c, y1.data(), t.data(), w.data(), st)) != cudaSuccess) return e;
            comb(sum, 1.0, sum.data(), 1.0, w.data());
            std::vector<void*> lv(lam, lam + nb);
            comb(lv, 1.0, lam, 1.0, sum.data());
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_rk4_adjoint(DevCtx& c, void* const* u0, void* const* lam, double dt, int nsteps, int every,
                               const std::vector<std::vector<void*>>& ck, const std::vector<std::vector<void*>>& blk,
                               const std::vector<std::vector<void*>>& tmp, cudaStream_t st) {
    return c.precision == 0 ? rk4_adjoint_impl<double>(c, u0, lam, dt, nsteps, every, ck, blk, tmp, st)
                            : rk4_adjoint_impl<float>(c, u0, lam, dt, nsteps, every, ck, blk, tmp, st);
}

}  // namespace fr
