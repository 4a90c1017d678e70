// Host-side set-up of the FR discretisation (Sec. 2, App. A).
//
// Everything here is evaluated in long double and rounded once to FP64:
//   * Gauss-Legendre points by Newton iteration on P_n;
//   * nodal bases: for tensor elements the product of 1D Lagrange polynomials
//     through the Gauss-Legendre points (the Vandermonde construction of Sec. 2
//     with a tensor Lagrange spanning set gives exactly this); for triangles a
//     monomial Vandermonde matrix inverted by Gauss-Jordan elimination;
//   * correction functions: for tensor elements the derivative of the right
//     VCJH correction function g_R = (P_p + (eta P_{p-1} + P_{p+1})/(1+eta))/2
//     (eta = 0: DG, the right Radau polynomial; p/(p+1): SD; (p+1)/p: HU)
//     times the tangential Lagrange factors; for triangles (DG only) the lift
//     of the face Lagrange polynomial through the exact (collapsed-Gauss)
//     mass matrix;
//   * metric terms from the Lagrange shape functions of each element.
#include "fr_host.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace fr {

using ldbl = long double;

// ------------------------------------------------------------ 1D polynomials
static void legendre_pd(int n, ldbl x, ldbl& p, ldbl& dp) {
    if (n == 0) { p = 1; dp = 0; return; }
    ldbl pm = 1, pc = x, dm = 0, dc = 1;
    for (int k = 1; k < n; ++k) {
        ldbl pn = ((2 * k + 1) * x * pc - k * pm) / (k + 1);
        ldbl dn = dm + (2 * k + 1) * pc;          // P'_{k+1} = P'_{k-1} + (2k+1) P_k
        pm = pc; pc = pn; dm = dc; dc = dn;
    }
    p = pc; dp = dc;
}

static void gauss_legendre(int n, std::vector<ldbl>& x, std::vector<ldbl>& w) {
    x.assign(n, 0); w.assign(n, 0);
    const ldbl pi = acosl(-1.0L);
    for (int i = 0; i < n; ++i) {
        ldbl z = cosl(pi * (i + 0.75L) / (n + 0.5L));
        for (int it = 0; it < 100; ++it) {
            ldbl p, dp;
            legendre_pd(n, z, p, dp);
            ldbl dz = p / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        ldbl p, dp;
        legendre_pd(n, z, p, dp);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2 / ((1 - z * z) * dp * dp);
    }
}

static void lagrange1d(const ldbl* nodes, int n, ldbl x, ldbl* L, ldbl* dL) {
    for (int j = 0; j < n; ++j) {
        ldbl v = 1, d = 0;
        for (int m = 0; m < n; ++m) {
            if (m == j) continue;
            ldbl den = nodes[j] - nodes[m];
            d = d * (x - nodes[m]) / den + v / den;
            v = v * (x - nodes[m]) / den;
        }
        L[j] = v;
        if (dL) dL[j] = d;
    }
}

// Gauss-Jordan inverse with partial pivoting (n x n, row-major, in place).
static bool invert(std::vector<ldbl>& A, int n) {
    std::vector<ldbl> I(n * n, 0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
        if (fabsl(A[piv * n + c]) < 1e-300L) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[c * n + k], A[piv * n + k]);
                std::swap(I[c * n + k], I[piv * n + k]);
            }
        ldbl d = A[c * n + c];
        for (int k = 0; k < n; ++k) { A[c * n + k] /= d; I[c * n + k] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            ldbl f = A[r * n + c];
            if (f == 0) continue;
            for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
        }
    }
    A.swap(I);
    return true;
}

// ------------------------------------------------------------ faces
static int ndims_of(int et) { return et == ET_HEX ? 3 : 2; }
static int nfaces_of(int et) { return et == ET_QUAD ? 4 : (et == ET_TRI ? 3 : 6); }

// map from face parameters to reference coordinates; also unit normal and
// reference measure per unit parameter measure
static void face_info(int et, int f, ldbl* n, ldbl& dsdt) {
    dsdt = 1;
    for (int i = 0; i < 3; ++i) n[i] = 0;
    if (et == ET_QUAD) {
        static const int nx[4] = {0, 1, 0, -1}, ny[4] = {-1, 0, 1, 0};
        n[0] = nx[f]; n[1] = ny[f];
    } else if (et == ET_TRI) {
        if (f == 0) { n[1] = -1; }
        else if (f == 1) { n[0] = n[1] = 1 / sqrtl(2.0L); dsdt = sqrtl(2.0L); }
        else { n[0] = -1; }
    } else {
        static const int ax[6] = {2, 1, 0, 1, 0, 2}, sg[6] = {-1, -1, 1, 1, -1, 1};
        n[ax[f]] = sg[f];
    }
}

void face_point(int et, int f, const ldbl* par, ldbl* x) {
    if (et == ET_QUAD) {
        ldbl t = par[0];
        switch (f) {
            case 0: x[0] = t; x[1] = -1; break;
            case 1: x[0] = 1; x[1] = t; break;
            case 2: x[0] = -t; x[1] = 1; break;
            default: x[0] = -1; x[1] = -t; break;
        }
    } else if (et == ET_TRI) {
        ldbl t = par[0];
        switch (f) {
            case 0: x[0] = t; x[1] = -1; break;
            case 1: x[0] = -t; x[1] = t; break;
            default: x[0] = -1; x[1] = -t; break;
        }
    } else {
        static const int ax[6] = {2, 1, 0, 1, 0, 2}, sg[6] = {-1, -1, 1, 1, -1, 1};
        int a = ax[f], k = 0;
        for (int i = 0; i < 3; ++i) {
            if (i == a) x[i] = sg[f];
            else x[i] = par[k++];
        }
    }
}

// ------------------------------------------------------------ nodal basis
static void tri_monomials(int p, const ldbl* x, ldbl* m, ldbl* dm /*[2][nb]*/) {
    int k = 0, nb = (p + 1) * (p + 2) / 2;
    for (int b = 0; b <= p; ++b)
        for (int a = 0; a + b <= p; ++a, ++k) {
            ldbl xa = powl(x[0], a), yb = powl(x[1], b);
            m[k] = xa * yb;
            if (dm) {
                dm[k] = a > 0 ? a * powl(x[0], a - 1) * yb : 0;
                dm[nb + k] = b > 0 ? b * xa * powl(x[1], b - 1) : 0;
            }
        }
}

void ElemType::nodal(const ldbl* x, ldbl* val, ldbl* grad) const {
    if (etype == ET_TRI) {
        int nb = nupts;
        std::vector<ldbl> m(nb), dm(2 * nb);
        tri_monomials(p, x, m.data(), dm.data());
        for (int r = 0; r < nupts; ++r) {
            ldbl v = 0, g0 = 0, g1 = 0;
            for (int k = 0; k < nb; ++k) {
                ldbl c = tri_coef[k * nupts + r];
                v += c * m[k]; g0 += c * dm[k]; g1 += c * dm[nb + k];
            }
            val[r] = v;
            if (grad) { grad[r] = g0; grad[nupts + r] = g1; }
        }
        return;
    }
    int n1 = p + 1;
    std::vector<ldbl> nodes(gl.begin(), gl.end());
    ldbl L[3][16], dL[3][16];
    for (int d = 0; d < ndims; ++d) lagrange1d(nodes.data(), n1, x[d], L[d], dL[d]);
    for (int r = 0; r < nupts; ++r) {
        int idx[3] = {r % n1, (r / n1) % n1, r / (n1 * n1)};
        ldbl v = 1;
        for (int d = 0; d < ndims; ++d) v *= L[d][idx[d]];
        val[r] = v;
        if (grad)
            for (int dd = 0; dd < ndims; ++dd) {
                ldbl g = 1;
                for (int d = 0; d < ndims; ++d) g *= (d == dd ? dL[d][idx[d]] : L[d][idx[d]]);
                grad[dd * nupts + r] = g;
            }
    }
}

bool build_element(int et, int p, ElemType& el, std::string& err, int correction) {
    if (p < 1 || p > 10) { err = "order must be in [1, 10]"; return false; }
    if (correction < 0 || correction > 2) { err = "correction must be 0 (DG), 1 (SD) or 2 (HU)"; return false; }
    if (et == ET_TRI && correction != 0) { err = "SD / HU correction functions need a tensor element"; return false; }
    const ldbl eta = correction == 0 ? 0.0L : correction == 1 ? (ldbl)p / (p + 1) : (ldbl)(p + 1) / p;
    el = ElemType();
    el.etype = et; el.p = p;
    el.ndims = ndims_of(et);
    el.nfaces = nfaces_of(et);
    int d = el.ndims, n1 = p + 1;
    std::vector<ldbl> g, w;
    gauss_legendre(n1, g, w);
    el.gl.assign(g.begin(), g.end());
    el.glw.assign(w.begin(), w.end());
    // solution points
    std::vector<ldbl> up;
    if (et == ET_QUAD) {
        for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) { up.push_back(g[i]); up.push_back(g[j]); }
    } else if (et == ET_HEX) {
        for (int k = 0; k < n1; ++k) for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
            up.push_back(g[i]); up.push_back(g[j]); up.push_back(g[k]);
        }
    } else {
        for (int j = 0; j <= p; ++j) for (int i = 0; i + j <= p; ++i) {
            up.push_back(-1 + 2.0L * (i + 1) / (p + 3));
            up.push_back(-1 + 2.0L * (j + 1) / (p + 3));
        }
    }
    el.nupts = (int)(up.size() / d);
    int nu = el.nupts;
    // flux points
    el.nfp_face = d == 2 ? n1 : n1 * n1;
    std::vector<ldbl> fp, fn;
    for (int f = 0; f < el.nfaces; ++f) {
        ldbl nrm[3], dsdt;
        face_info(et, f, nrm, dsdt);
        for (int k = 0; k < el.nfp_face; ++k) {
            ldbl par[2] = {g[k % n1], d == 3 ? g[k / n1] : 0}, x[3];
            face_point(et, f, par, x);
            for (int i = 0; i < d; ++i) { fp.push_back(x[i]); fn.push_back(nrm[i]); }
            el.fface.push_back(f);
        }
    }
    el.nfpts = (int)el.fface.size();
    int nf = el.nfpts;
    el.upts.assign(up.begin(), up.end());
    el.fpts.assign(fp.begin(), fp.end());
    el.fnorm.assign(fn.begin(), fn.end());
    // triangle: monomial Vandermonde, Vm[sigma][k] = m_k(x_sigma); coef = Vm^{-1}
    if (et == ET_TRI) {
        std::vector<ldbl> Vm(nu * nu), m(nu);
        for (int s = 0; s < nu; ++s) {
            tri_monomials(p, &up[s * 2], m.data(), nullptr);
            for (int k = 0; k < nu; ++k) Vm[s * nu + k] = m[k];
        }
        if (!invert(Vm, nu)) { err = "singular triangle Vandermonde"; return false; }
        el.tri_coef = Vm;   // coef[k][rho]
    }
    // operators in long double
    std::vector<ldbl> M0(nf * nu), M1(nu * d * nu), M2(nf * d * nu), M3(nu * nf, 0),
        M4(d * nu * nu), M6(d * nu * nf);
    std::vector<ldbl> val(nu), grd(d * nu);
    for (int s = 0; s < nf; ++s) {
        el.nodal(&fp[s * d], val.data(), nullptr);
        for (int r = 0; r < nu; ++r) {
            M0[s * nu + r] = val[r];
            for (int i = 0; i < d; ++i) M2[s * d * nu + i * nu + r] = val[r] * fn[s * d + i];
        }
    }
    for (int s = 0; s < nu; ++s) {
        el.nodal(&up[s * d], val.data(), grd.data());
        for (int i = 0; i < d; ++i)
            for (int r = 0; r < nu; ++r) {
                M4[(i * nu + s) * nu + r] = grd[i * nu + r];
                M1[s * d * nu + i * nu + r] = grd[i * nu + r];
            }
    }
    // correction functions (DG)
    if (et != ET_TRI) {
        for (int s = 0; s < nf; ++s) {
            int ax = 0;
            for (int i = 0; i < d; ++i) if (fabsl(fn[s * d + i]) > 0.5L) ax = i;
            ldbl sg = fn[s * d + ax] > 0 ? 1 : -1;
            for (int r = 0; r < nu; ++r) {
                ldbl xs = sg * up[r * d + ax], p0, d0, p1, d1, pm, dm;
                legendre_pd(p, xs, p0, d0);
                legendre_pd(p + 1, xs, p1, d1);
                legendre_pd(p - 1, xs, pm, dm);
                ldbl v = 0.5L * (d0 + (eta * dm + d1) / (1.0L + eta));   // g_R'(xs)
                for (int k = 0; k < d; ++k) {
                    if (k == ax) continue;
                    ldbl L[16];
                    lagrange1d(g.data(), n1, up[r * d + k], L, nullptr);
                    int j = 0;
                    for (int q = 1; q < n1; ++q)
                        if (fabsl(g[q] - fp[s * d + k]) < fabsl(g[j] - fp[s * d + k])) j = q;
                    v *= L[j];
                }
                M3[r * nf + s] = v;
            }
        }
    } else {
        // lift: Mass M3 = E with exact collapsed-Gauss mass matrix
        int nq = p + 3;
        std::vector<ldbl> qx, qw;
        gauss_legendre(nq, qx, qw);
        std::vector<ldbl> mass(nu * nu, 0), E(nu * nf, 0);
        for (int ia = 0; ia < nq; ++ia)
            for (int ib = 0; ib < nq; ++ib) {
                ldbl a = qx[ia], b = qx[ib];
                ldbl x[2] = {(1 + a) * (1 - b) / 2 - 1, b};
                ldbl wt = qw[ia] * qw[ib] * (1 - b) / 2;
                el.nodal(x, val.data(), nullptr);
                for (int i = 0; i < nu; ++i)
                    for (int j = 0; j < nu; ++j) mass[i * nu + j] += wt * val[i] * val[j];
            }
        for (int f = 0; f < 3; ++f) {
            ldbl nrm[3], dsdt;
            face_info(et, f, nrm, dsdt);
            for (int q = 0; q < nq; ++q) {
                ldbl x[2], par[1] = {qx[q]};
                face_point(et, f, par, x);
                el.nodal(x, val.data(), nullptr);
                ldbl L[16];
                lagrange1d(g.data(), n1, qx[q], L, nullptr);
                for (int k = 0; k < n1; ++k) {
                    int s = f * n1 + k;
                    for (int i = 0; i < nu; ++i) E[i * nf + s] += qw[q] * dsdt * val[i] * L[k];
                }
            }
        }
        if (!invert(mass, nu)) { err = "singular mass matrix"; return false; }
        for (int i = 0; i < nu; ++i)
            for (int s = 0; s < nf; ++s) {
                ldbl acc = 0;
                for (int k = 0; k < nu; ++k) acc += mass[i * nu + k] * E[k * nf + s];
                M3[i * nf + s] = acc;
            }
    }
    for (int i = 0; i < d; ++i)
        for (int s = 0; s < nu; ++s)
            for (int r = 0; r < nf; ++r) M6[(i * nu + s) * nf + r] = fn[r * d + i] * M3[s * nf + r];
    // fused forms of App. A
    std::vector<ldbl> M46(d * nu * nu), M132(nu * d * nu);
    for (int a = 0; a < d * nu; ++a)
        for (int r = 0; r < nu; ++r) {
            ldbl acc = M4[a * nu + r];
            for (int s = 0; s < nf; ++s) acc -= M6[a * nf + s] * M0[s * nu + r];
            M46[a * nu + r] = acc;
        }
    for (int r = 0; r < nu; ++r)
        for (int a = 0; a < d * nu; ++a) {
            ldbl acc = M1[r * d * nu + a];
            for (int s = 0; s < nf; ++s) acc -= M3[r * nf + s] * M2[s * d * nu + a];
            M132[r * d * nu + a] = acc;
        }
    auto cp = [](const std::vector<ldbl>& a, std::vector<double>& b) { b.assign(a.begin(), a.end()); };
    cp(M0, el.M0); cp(M1, el.M1); cp(M2, el.M2); cp(M3, el.M3); cp(M4, el.M4); cp(M6, el.M6);
    cp(M46, el.M46); cp(M132, el.M132);
    // solution-point quadrature weights on the reference element
    el.qw.assign(nu, 0.0);
    if (et != ET_TRI) {
        for (int r = 0; r < nu; ++r) {
            int idx[3] = {r % n1, (r / n1) % n1, r / (n1 * n1)};
            ldbl v = 1;
            for (int k = 0; k < d; ++k) v *= w[idx[k]];
            el.qw[r] = (double)v;
        }
    } else {
        int nq = p + 3;
        std::vector<ldbl> qx, qwt, acc(nu, 0);
        gauss_legendre(nq, qx, qwt);
        for (int ia = 0; ia < nq; ++ia)
            for (int ib = 0; ib < nq; ++ib) {
                ldbl a = qx[ia], b = qx[ib];
                ldbl x[2] = {(1 + a) * (1 - b) / 2 - 1, b};
                el.nodal(x, val.data(), nullptr);
                for (int i = 0; i < nu; ++i) acc[i] += qwt[ia] * qwt[ib] * (1 - b) / 2 * val[i];
            }
        for (int i = 0; i < nu; ++i) el.qw[i] = (double)acc[i];
    }
    return true;
}

// ------------------------------------------------------------ element mappings
bool shape_functions(int et, int nn, const ldbl* x, ldbl* N, ldbl* dN) {
    if (et == ET_QUAD || et == ET_HEX) {
        int d = ndims_of(et);
        int m = (et == ET_QUAD) ? (nn == 4 ? 2 : (nn == 9 ? 3 : 0)) : (nn == 8 ? 2 : (nn == 27 ? 3 : 0));
        if (!m) return false;
        ldbl eq[3];
        if (m == 2) { eq[0] = -1; eq[1] = 1; } else { eq[0] = -1; eq[1] = 0; eq[2] = 1; }
        ldbl L[3][3], dL[3][3];
        for (int k = 0; k < d; ++k) lagrange1d(eq, m, x[k], L[k], dL[k]);
        for (int a = 0; a < nn; ++a) {
            int idx[3] = {a % m, (a / m) % m, a / (m * m)};
            ldbl v = 1;
            for (int k = 0; k < d; ++k) v *= L[k][idx[k]];
            N[a] = v;
            for (int dd = 0; dd < d; ++dd) {
                ldbl gg = 1;
                for (int k = 0; k < d; ++k) gg *= (k == dd ? dL[k][idx[k]] : L[k][idx[k]]);
                dN[dd * nn + a] = gg;
            }
        }
        return true;
    }
    if (et == ET_TRI) {
        ldbl l[3] = {-(x[0] + x[1]) / 2, (1 + x[0]) / 2, (1 + x[1]) / 2};
        const ldbl dl[2][3] = {{-0.5L, 0.5L, 0}, {-0.5L, 0, 0.5L}};
        if (nn == 3) {
            for (int a = 0; a < 3; ++a) { N[a] = l[a]; dN[a] = dl[0][a]; dN[3 + a] = dl[1][a]; }
            return true;
        }
        if (nn == 6) {
            static const int pa[3] = {0, 1, 2}, pb[3] = {1, 2, 0};
            for (int a = 0; a < 3; ++a) {
                N[a] = l[a] * (2 * l[a] - 1);
                for (int dd = 0; dd < 2; ++dd) dN[dd * 6 + a] = dl[dd][a] * (4 * l[a] - 1);
            }
            for (int e = 0; e < 3; ++e) {
                int a = pa[e], b = pb[e];
                N[3 + e] = 4 * l[a] * l[b];
                for (int dd = 0; dd < 2; ++dd) dN[dd * 6 + 3 + e] = 4 * (dl[dd][a] * l[b] + l[a] * dl[dd][b]);
            }
            return true;
        }
    }
    return false;
}

bool prepare_block(HostBlock& blk) {
    const ElemType& el = *blk.el;
    int d = el.ndims, nn = blk.nnodes;
    ldbl N[27], dN[81];
    auto fill = [&](const std::vector<double>& pts, int np, std::vector<double>& Nt, std::vector<double>& dNt) {
        Nt.assign((size_t)np * nn, 0.0);
        dNt.assign((size_t)np * d * nn, 0.0);
        for (int s = 0; s < np; ++s) {
            ldbl x[3] = {0, 0, 0};
            for (int i = 0; i < d; ++i) x[i] = pts[s * d + i];
            if (!shape_functions(blk.etype, nn, x, N, dN)) return false;
            for (int a = 0; a < nn; ++a) {
                Nt[(size_t)s * nn + a] = (double)N[a];
                for (int j = 0; j < d; ++j) dNt[((size_t)s * d + j) * nn + a] = (double)dN[j * nn + a];
            }
        }
        return true;
    };
    if (!fill(el.upts, el.nupts, blk.Nu, blk.dNu)) return false;
    if (!fill(el.fpts, el.nfpts, blk.Nf, blk.dNf)) return false;
    blk.Nc.assign((size_t)el.nfaces * nn, 0.0);
    for (int f = 0; f < el.nfaces; ++f) {
        ldbl par[2] = {0, 0}, x[3] = {0, 0, 0};
        face_point(blk.etype, f, par, x);
        if (!shape_functions(blk.etype, nn, x, N, dN)) return false;
        for (int a = 0; a < nn; ++a) blk.Nc[(size_t)f * nn + a] = (double)N[a];
    }
    return true;
}

// J[i][j] = d x_i / d xi_j and X at table point s (dN: [npts][d][nn])
static void jacobian_tab(const HostBlock& blk, int64_t e, const double* Nt, const double* dNt, int s,
                         double J[3][3], double* X) {
    int d = blk.el->ndims, nn = blk.nnodes;
    const double* nd = &blk.nodes[(size_t)e * nn * d];
    const double* dn = dNt + (size_t)s * d * nn;
    for (int i = 0; i < d; ++i) {
        if (X) {
            double acc = 0;
            for (int a = 0; a < nn; ++a) acc += Nt[(size_t)s * nn + a] * nd[a * d + i];
            X[i] = acc;
        }
        for (int j = 0; j < d; ++j) {
            double acc = 0;
            for (int a = 0; a < nn; ++a) acc += dn[j * nn + a] * nd[a * d + i];
            J[i][j] = acc;
        }
    }
}

static double adjugate(int d, const double J[3][3], double A[3][3]) {
    if (d == 2) {
        A[0][0] = J[1][1]; A[0][1] = -J[0][1];
        A[1][0] = -J[1][0]; A[1][1] = J[0][0];
        return J[0][0] * J[1][1] - J[0][1] * J[1][0];
    }
    A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

bool element_metrics(const HostBlock& blk, int64_t e, double* adj, double* det) {
    const ElemType& el = *blk.el;
    int d = el.ndims;
    bool ok = true;
    for (int s = 0; s < el.nupts; ++s) {
        double J[3][3], A[3][3];
        jacobian_tab(blk, e, blk.Nu.data(), blk.dNu.data(), s, J, nullptr);
        double dt = adjugate(d, J, A);
        if (!(dt > 0)) ok = false;
        det[s] = dt;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) adj[(s * d + i) * d + j] = A[i][j];
    }
    return ok;
}

// physical coords, unit normal and magnitude at flux point s of element e
static bool fpt_geometry(const HostBlock& blk, int64_t e, int s, double* X, double* nrm, double& mag) {
    const ElemType& el = *blk.el;
    int d = el.ndims;
    double J[3][3], A[3][3];
    jacobian_tab(blk, e, blk.Nf.data(), blk.dNf.data(), s, J, X);
    double dt = adjugate(d, J, A);
    double v[3] = {0, 0, 0}, m2 = 0;
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j < d; ++j) v[i] += A[j][i] * el.fnorm[s * d + j];   // adj(J)^T n
        m2 += v[i] * v[i];
    }
    double m = std::sqrt(m2);
    for (int i = 0; i < d; ++i) nrm[i] = v[i] / m;
    for (int i = d; i < 3; ++i) nrm[i] = 0;
    mag = m;
    return dt > 0;
}

// ------------------------------------------------------------ pairing
namespace {
struct Face { int32_t b, f; int64_t n; double c[3]; };

inline uint64_t cell_key(const int64_t* k) {
    const int64_t off = 1 << 20;
    return ((uint64_t)(k[0] + off) << 42) | ((uint64_t)(k[1] + off) << 21) | (uint64_t)(k[2] + off);
}
}  // namespace

bool pair_mesh(int d, const std::vector<HostBlock>& blocks, const int64_t* bfaces, int64_t nbfaces,
               const double* periodic, int nper, std::vector<HostPair>& pairs, std::vector<HostBnd>& bnds,
               std::string& err) {
    // 1. faces and their centres (face-parameter origin mapped to physical space)
    std::vector<int64_t> foff(blocks.size() + 1, 0);
    for (size_t b = 0; b < blocks.size(); ++b) foff[b + 1] = foff[b] + blocks[b].nelem * blocks[b].el->nfaces;
    int64_t nface = foff.back();
    std::vector<Face> faces(nface);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t b = 0; b < blocks.size(); ++b) {
        const HostBlock& blk = blocks[b];
        for (size_t k = 0; k < blk.nodes.size(); ++k) {
            int i = k % d;
            lo[i] = std::min(lo[i], blk.nodes[k]);
            hi[i] = std::max(hi[i], blk.nodes[k]);
        }
    }
    double ext = 1.0;
    for (int i = 0; i < d; ++i) ext = std::max(ext, hi[i] - lo[i]);
    const double tol = 1e-8 * ext, cell = 1e-5 * ext;
    for (size_t b = 0; b < blocks.size(); ++b) {
        const HostBlock& blk = blocks[b];
        int nfc = blk.el->nfaces;
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < blk.nelem; ++e)
            for (int f = 0; f < nfc; ++f) {
                Face& F = faces[foff[b] + e * nfc + f];
                F.b = (int32_t)b; F.n = e; F.f = f;
                const double* nd = &blk.nodes[(size_t)e * blk.nnodes * d];
                for (int i = 0; i < 3; ++i) {
                    double acc = 0;
                    if (i < d)
                        for (int a = 0; a < blk.nnodes; ++a) acc += blk.Nc[(size_t)f * blk.nnodes + a] * nd[a * d + i];
                    F.c[i] = acc;
                }
            }
    }
    // 2. spatial hash (sorted cell keys)
    std::vector<std::pair<uint64_t, int64_t>> keys(nface);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nface; ++i) {
        int64_t k[3] = {0, 0, 0};
        for (int j = 0; j < d; ++j) k[j] = (int64_t)std::floor((faces[i].c[j] - lo[j]) / cell);
        keys[i] = {cell_key(k), i};
    }
    std::sort(keys.begin(), keys.end());
    // shifts: every combination of -1/0/+1 times each periodic vector (zero first)
    std::vector<std::array<double, 3>> shifts;
    int ncomb = 1;
    for (int i = 0; i < nper; ++i) ncomb *= 3;
    for (int c = 0; c < ncomb; ++c) {
        std::array<double, 3> s = {0, 0, 0};
        int cc = c;
        for (int i = 0; i < nper; ++i) {
            int m = cc % 3; cc /= 3;
            double fac = m == 0 ? 0.0 : (m == 1 ? 1.0 : -1.0);
            for (int j = 0; j < d; ++j) s[j] += fac * periodic[i * d + j];
        }
        shifts.push_back(s);
    }
    std::vector<int64_t> match(nface, -1);
    std::vector<int32_t> mshift(nface, -1);
    bool dup = false;
#pragma omp parallel for schedule(dynamic, 4096) reduction(|| : dup)
    for (int64_t i = 0; i < nface; ++i) {
        const Face& A = faces[i];
        int found = 0;
        for (size_t s = 0; s < shifts.size() && !found; ++s) {
            double t[3] = {0, 0, 0};
            for (int j = 0; j < d; ++j) t[j] = A.c[j] + shifts[s][j];
            // cells within tol of the target in every direction
            int64_t lo_k[3] = {0, 0, 0}, hi_k[3] = {0, 0, 0};
            for (int j = 0; j < d; ++j) {
                lo_k[j] = (int64_t)std::floor((t[j] - tol - lo[j]) / cell);
                hi_k[j] = (int64_t)std::floor((t[j] + tol - lo[j]) / cell);
            }
            for (int64_t kx = lo_k[0]; kx <= hi_k[0]; ++kx)
                for (int64_t ky = lo_k[1]; ky <= hi_k[1]; ++ky)
                    for (int64_t kz = lo_k[2]; kz <= hi_k[2]; ++kz) {
                        int64_t k[3] = {kx, ky, kz};
                        uint64_t key = cell_key(k);
                        auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(key, (int64_t)-1));
                        for (; it != keys.end() && it->first == key; ++it) {
                            int64_t j = it->second;
                            if (j == i) continue;
                            double dist = 0;
                            for (int q = 0; q < d; ++q) dist += (faces[j].c[q] - t[q]) * (faces[j].c[q] - t[q]);
                            if (std::sqrt(dist) < tol) {
                                if (found && match[i] != j) dup = true;
                                match[i] = j; mshift[i] = (int32_t)s; found = 1;
                            }
                        }
                    }
        }
    }
    if (dup) { err = "a face matched more than one face"; return false; }
    // 3. boundary faces
    std::vector<int32_t> btype(nface, -1);
    for (int64_t k = 0; k < nbfaces; ++k) {
        int64_t b = bfaces[4 * k], e = bfaces[4 * k + 1], f = bfaces[4 * k + 2], t = bfaces[4 * k + 3];
        if (b < 0 || b >= (int64_t)blocks.size() || e < 0 || e >= blocks[b].nelem || f < 0 ||
            f >= blocks[b].el->nfaces || t < 0 || t > 3) {
            err = "bad boundary face entry"; return false;
        }
        btype[foff[b] + e * blocks[b].el->nfaces + f] = (int32_t)t;
    }
    int64_t npairf = 0, nbf = 0;
    for (int64_t i = 0; i < nface; ++i) {
        if (match[i] >= 0 && btype[i] >= 0) { err = "boundary face is also paired"; return false; }
        if (match[i] < 0 && btype[i] < 0) {
            err = "unmatched face (block " + std::to_string(faces[i].b) + ", element " +
                  std::to_string(faces[i].n) + ", face " + std::to_string(faces[i].f) + ")";
            return false;
        }
        if (match[i] >= 0 && match[match[i]] != i) { err = "asymmetric face match"; return false; }
        if (match[i] > i) ++npairf;
        if (btype[i] >= 0) ++nbf;
    }
    // 4. flux-point pairs of every matched face pair (L = lower face index)
    std::vector<int64_t> plist;
    plist.reserve(npairf);
    for (int64_t i = 0; i < nface; ++i) if (match[i] > i) plist.push_back(i);
    int nfp = blocks.empty() ? 0 : blocks[0].el->nfp_face;
    pairs.assign((size_t)npairf * nfp, HostPair());
    bool bad = false;
#pragma omp parallel for schedule(static) reduction(|| : bad)
    for (int64_t q = 0; q < npairf; ++q) {
        int64_t i = plist[q], j = match[i];
        const Face &A = faces[i], &B = faces[j];
        const HostBlock &bA = blocks[A.b], &bB = blocks[B.b];
        const auto& sh = shifts[mshift[i]];
        double XA[128][3], XB[128][3], nA[128][3], nB[128][3], mA[128], mB[128];
        int sA = A.f * nfp, sB = B.f * nfp;
        for (int k = 0; k < nfp; ++k) {
            if (!fpt_geometry(bA, A.n, sA + k, XA[k], nA[k], mA[k])) bad = true;
            if (!fpt_geometry(bB, B.n, sB + k, XB[k], nB[k], mB[k])) bad = true;
        }
        for (int k = 0; k < nfp; ++k) {
            int hit = -1;
            for (int m = 0; m < nfp; ++m) {
                double dist = 0;
                for (int c = 0; c < d; ++c) dist += (XA[k][c] + sh[c] - XB[m][c]) * (XA[k][c] + sh[c] - XB[m][c]);
                if (std::sqrt(dist) < tol) { if (hit >= 0) bad = true; hit = m; }
            }
            if (hit < 0) { bad = true; continue; }
            HostPair& P = pairs[q * nfp + k];
            P.bL = A.b; P.fL = sA + k; P.nL = A.n;
            P.bR = B.b; P.fR = sB + hit; P.nR = B.n;
            for (int c = 0; c < 3; ++c) P.nrm[c] = nA[k][c];
            P.magL = mA[k]; P.magR = mB[hit];
        }
    }
    if (bad) { err = "flux points of a matched face pair do not coincide (or non-positive Jacobian)"; return false; }
    bnds.clear();
    bnds.reserve((size_t)nbf * nfp);
    for (int64_t i = 0; i < nface; ++i) {
        if (btype[i] < 0) continue;
        const Face& A = faces[i];
        const HostBlock& bA = blocks[A.b];
        for (int k = 0; k < nfp; ++k) {
            HostBnd Bd;
            double X[3];
            Bd.b = A.b; Bd.n = A.n; Bd.f = A.f * nfp + k; Bd.bctype = btype[i];
            if (!fpt_geometry(bA, A.n, Bd.f, X, Bd.nrm, Bd.mag)) { err = "non-positive Jacobian at boundary"; return false; }
            bnds.push_back(Bd);
        }
    }
    return true;
}

}  // namespace fr
