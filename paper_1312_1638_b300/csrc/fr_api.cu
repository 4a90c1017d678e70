// C ABI of the FR library: context set-up (host work + device upload) and the
// stream-ordered entry points declared in include/fr.h.
#include <algorithm>
#include <cmath>
#include <array>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fr.h"
#include "fr_dev.hpp"
#include "fr_host.hpp"
#include "fr_tc.hpp"

struct fr_ctx {
    std::string err;
    fr_params prm{};
    int ndims = 0, nvars = 0;
    std::vector<std::unique_ptr<fr::ElemType>> etypes;
    std::vector<fr::HostBlock> hblocks;
    std::vector<fr::HostPair> pairs;     // interior flux-point pairs (sorted like the device tables)
    std::vector<fr::HostBnd> bnds;       // boundary flux points
    fr::DevCtx dev;
    std::vector<void*> allocs;
    // CUDA graph of one RK4 step, replayed by fr_rk4 (keyed by state pointers and dt)
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t rk_exec = nullptr;
    std::vector<void*> rk_ptrs;
    double rk_dt = 0.0;
    // partitioned context (fr_setup_part): this rank, the number of ranks, the
    // neighbour ranks and, per neighbour, the key (global L block, element,
    // flux point) of every exchange slot
    int part_rank = -1, part_n = 0;
    std::vector<int> nbr_q;
    std::vector<std::vector<std::array<int64_t, 3>>> nbr_keys;
    cudaStream_t xstream = nullptr;     // exchange copies (fr_rhs_parts, owned by rank 0's context)
    cudaEvent_t xev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {
// one cross-partition flux-point pair seen from this rank
struct MpiPair {
    int q;                   // neighbour rank
    int b;                   // my (local) block
    int32_t f;               // my flux point
    int64_t n;               // my local element
    bool mine_L;             // my side is the global L side
    std::array<int64_t, 3> key;   // global L side (block, element, flux point)
    double nrm[3], magL, magR;
};
}  // namespace

static thread_local std::string g_setup_err;

namespace {

struct Fail {
    fr_status st;
    std::string msg;
};

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw Fail{e_ == cudaErrorMemoryAllocation ? FR_ERR_OOM : FR_ERR_CUDA,           \
                       std::string(#call) + ": " + cudaGetErrorString(e_)};                   \
    } while (0)

void* dalloc(fr_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    CK(cudaMalloc(&p, bytes));
    c->allocs.push_back(p);
    return p;
}

template <typename T>
void* upload(fr_ctx* c, const std::vector<T>& h) {
    void* p = dalloc(c, h.size() * sizeof(T));
    CK(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

// convert a double vector to the compute type and upload
void* upload_real(fr_ctx* c, const std::vector<double>& h, bool fp64) {
    if (fp64) return upload(c, h);
    std::vector<float> f(h.begin(), h.end());
    return upload(c, f);
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// the rows' nonzeros (column, value) as [rows][nnz] packed entries in the
// compute type, each row zero-padded with (value 0, column 0)
template <typename T>
static void* upload_pairs_t(fr_ctx* c, const std::vector<std::vector<std::pair<int, double>>>& rows, int nnz) {
    std::vector<fr::SpPair<T>> e(rows.size() * (size_t)nnz, fr::SpPair<T>{T(0), 0});
    for (size_t r = 0; r < rows.size(); ++r)
        for (size_t j = 0; j < rows[r].size(); ++j) e[r * nnz + j] = fr::SpPair<T>{(T)rows[r][j].second, rows[r][j].first};
    return upload(c, e);
}

void* upload_pairs(fr_ctx* c, const std::vector<std::vector<std::pair<int, double>>>& rows, int nnz, bool fp64) {
    return fp64 ? upload_pairs_t<double>(c, rows, nnz) : upload_pairs_t<float>(c, rows, nnz);
}

// the nonzeros (column, value) of every row of a rows x cols row-major
// operator; entries below 1e-15 of their row's largest are the rounding of a
// vanishing Lagrange factor and are dropped.  *nnz: the most in any row.
static std::vector<std::vector<std::pair<int, double>>> nonzero_rows(const std::vector<double>& A, int64_t rows,
                                                                      int64_t cols, int* nnz) {
    std::vector<std::vector<std::pair<int, double>>> nz((size_t)rows);
    *nnz = 0;
    for (int64_t r = 0; r < rows; ++r) {
        double mx = 0;
        for (int64_t k = 0; k < cols; ++k) mx = std::max(mx, std::fabs(A[(size_t)(r * cols + k)]));
        for (int64_t k = 0; k < cols; ++k) {
            const double v = A[(size_t)(r * cols + k)];
            if (std::fabs(v) > 1e-15 * mx) nz[r].push_back({(int)k, v});
        }
        *nnz = std::max(*nnz, (int)nz[r].size());
    }
    return nz;
}

// the same rows as [rows][nnz] column indices and values (compute type),
// zero-padded
static void upload_idx_val(fr_ctx* c, const std::vector<std::vector<std::pair<int, double>>>& nz, int nnz, bool fp64,
                           int** idx_out, void** val_out) {
    std::vector<int> idx(nz.size() * (size_t)nnz, 0);
    std::vector<double> val(nz.size() * (size_t)nnz, 0.0);
    for (size_t r = 0; r < nz.size(); ++r)
        for (size_t j = 0; j < nz[r].size(); ++j) {
            idx[r * nnz + j] = nz[r][j].first;
            val[r * nnz + j] = nz[r][j].second;
        }
    *idx_out = (int*)upload(c, idx);
    *val_out = upload_real(c, val, fp64);
}

fr_status set_err(fr_ctx* c, fr_status st, const std::string& m) {
    if (c) c->err = m;
    else g_setup_err = m;
    return st;
}

// [A | B] side by side: A is r x ka, B is r x kb, both row-major
std::vector<double> hcat(const std::vector<double>& A, int ka, const std::vector<double>& B, int kb, int rows) {
    std::vector<double> o((size_t)rows * (ka + kb));
    for (int i = 0; i < rows; ++i) {
        std::copy(&A[(size_t)i * ka], &A[(size_t)i * ka] + ka, &o[(size_t)i * (ka + kb)]);
        std::copy(&B[(size_t)i * kb], &B[(size_t)i * kb] + kb, &o[(size_t)i * (ka + kb) + ka]);
    }
    return o;
}

template <typename T>
void fill_metrics(fr_ctx* c, const fr::HostBlock& hb, fr::DevBlock& B, int d) {
    const fr::ElemType& el = *hb.el;
    const int64_t ld = B.ld, nu = el.nupts;
    std::vector<T> smat((size_t)d * d * nu * ld, T(0)), rcp((size_t)nu * ld, T(0));
    std::vector<double> wdet((size_t)nu * ld, 0.0);
    bool ok = true;
#pragma omp parallel reduction(&& : ok)
    {
        std::vector<double> adj((size_t)nu * d * d), det(nu);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < hb.nelem; ++e) {
            if (!fr::element_metrics(hb, e, adj.data(), det.data())) ok = false;
            for (int s = 0; s < nu; ++s) {
                for (int k = 0; k < d * d; ++k) smat[((size_t)k * nu + s) * ld + e] = (T)adj[(size_t)s * d * d + k];
                rcp[(size_t)s * ld + e] = (T)(1.0 / det[s]);
                wdet[(size_t)s * ld + e] = el.qw[s] * det[s];
            }
        }
    }
    if (!ok) throw Fail{FR_ERR_MESH, "non-positive Jacobian at a solution point"};
    B.smat = upload(c, smat);
    B.rcpdjac = upload(c, rcp);
    B.wdet = (double*)upload(c, wdet);
}

// Tensor-line form of the gradient and divergence operators (quadrilaterals,
// hexahedra; see the tensor-line kernels): the lines in the kernels'
// numbering (direction i, then the other indices, xi fastest), each line's
// two end flux points found by their reference coordinates (the xi_i = -1
// one first), and n x (n+2) line matrices taken from the first line.  The
// form is accepted only if it rebuilds every row of the dense operators to
// 1e-12 of the row's largest entry (so no line or direction differs and no
// entry is missed).
struct LineForm {
    int n = 0;
    bool grad = false, div = false, interp = false;
    std::vector<double> A, B, I0;
    std::vector<int> fl;
};

static LineForm line_form(const fr::ElemType& el, int d) {
    LineForm L;
    if (el.etype != fr::ET_QUAD && el.etype != fr::ET_HEX) return L;
    const int n = el.p + 1, nu = el.nupts, nf = el.nfpts;
    int NU = 1;
    for (int i = 0; i < d; ++i) NU *= n;
    if (NU != nu || n < 2 || n > 6) return L;
    const int NL = NU / n, NLT = d * NL;
    const double tol = 1e-12;
    for (int s = 0; s < nu; ++s) {                       // s = a + n b (+ n^2 c) at the GL nodes (a, b, c)
        int r = s;
        for (int j = 0; j < d; ++j) {
            if (std::fabs(el.upts[(size_t)s * d + j] - el.gl[r % n]) > tol) return L;
            r /= n;
        }
    }
    std::vector<std::vector<int>> pts(NLT, std::vector<int>(n));
    std::vector<int> dir(NLT), fl((size_t)NLT * 2, -1);
    for (int l = 0; l < NLT; ++l) {
        const int i = l / NL, m = l % NL;
        int base, stride;
        if (d == 2) {
            base = i == 0 ? m * n : m;
            stride = i == 0 ? 1 : n;
        } else {
            base = i == 0 ? m * n : (i == 1 ? m % n + n * n * (m / n) : m);
            stride = i == 0 ? 1 : (i == 1 ? n : n * n);
        }
        dir[l] = i;
        for (int q = 0; q < n; ++q) pts[l][q] = base + q * stride;
        for (int f = 0; f < nf; ++f) {
            bool on = true;
            for (int j = 0; j < d && on; ++j)
                if (j != i && std::fabs(el.fpts[(size_t)f * d + j] - el.upts[(size_t)pts[l][0] * d + j]) > tol) on = false;
            if (!on) continue;
            const double x = el.fpts[(size_t)f * d + i];
            const int e = std::fabs(x + 1) < tol ? 0 : (std::fabs(x - 1) < tol ? 1 : -1);
            if (e < 0 || fl[2 * l + e] >= 0) return L;
            fl[2 * l + e] = f;
        }
        if (fl[2 * l] < 0 || fl[2 * l + 1] < 0) return L;
    }
    const int w = n + 2;
    auto close = [&](const std::vector<double>& rec, const double* row, size_t len) {
        double mx = 0, df = 0;
        for (size_t k = 0; k < len; ++k) {
            mx = std::max(mx, std::fabs(row[k]));
            df = std::max(df, std::fabs(row[k] - rec[k]));
        }
        return df <= tol * mx;
    };
    // gradient: row (i, s) of [M6 | M4 - M6 M0] from line l through s along i
    {
        std::vector<double> A((size_t)n * w);
        for (int q = 0; q < n; ++q) {
            const size_t r = (size_t)dir[0] * nu + pts[0][q];
            for (int k = 0; k < n; ++k) A[(size_t)q * w + k] = el.M46[r * nu + pts[0][k]];
            for (int e = 0; e < 2; ++e) A[(size_t)q * w + n + e] = el.M6[r * nf + fl[e]];
        }
        bool ok = true;
        std::vector<double> rec(nf + nu);
        for (int l = 0; l < NLT && ok; ++l)
            for (int q = 0; q < n && ok; ++q) {
                const size_t r = (size_t)dir[l] * nu + pts[l][q];
                std::fill(rec.begin(), rec.end(), 0.0);
                for (int k = 0; k < n; ++k) rec[nf + pts[l][k]] = A[(size_t)q * w + k];
                for (int e = 0; e < 2; ++e) rec[fl[2 * l + e]] = A[(size_t)q * w + n + e];
                std::vector<double> row(nf + nu);
                for (int f = 0; f < nf; ++f) row[f] = el.M6[r * nf + f];
                for (int k = 0; k < nu; ++k) row[nf + k] = el.M46[r * nu + k];
                ok = close(rec, row.data(), row.size());
            }
        L.grad = ok;
        L.A = A;
    }
    // divergence: row s of [M3 | M1 - M3 M2], one line per direction through s
    {
        std::vector<double> B((size_t)n * w);
        for (int q = 0; q < n; ++q) {
            const size_t s = pts[0][q];
            for (int k = 0; k < n; ++k) B[(size_t)q * w + k] = el.M132[s * d * nu + (size_t)dir[0] * nu + pts[0][k]];
            for (int e = 0; e < 2; ++e) B[(size_t)q * w + n + e] = el.M3[s * nf + fl[e]];
        }
        std::vector<std::vector<double>> rec(nu, std::vector<double>(nf + (size_t)d * nu, 0.0));
        for (int l = 0; l < NLT; ++l)
            for (int q = 0; q < n; ++q) {
                std::vector<double>& rr = rec[pts[l][q]];
                for (int k = 0; k < n; ++k) rr[nf + (size_t)dir[l] * nu + pts[l][k]] += B[(size_t)q * w + k];
                for (int e = 0; e < 2; ++e) rr[fl[2 * l + e]] += B[(size_t)q * w + n + e];
            }
        bool ok = true;
        for (int s = 0; s < nu && ok; ++s) {
            std::vector<double> row(nf + (size_t)d * nu);
            for (int f = 0; f < nf; ++f) row[f] = el.M3[(size_t)s * nf + f];
            for (int k = 0; k < d * nu; ++k) row[nf + k] = el.M132[(size_t)s * d * nu + k];
            ok = close(rec[s], row.data(), row.size());
        }
        L.div = ok;
        L.B = B;
    }
    // interpolation: row f of M0 for the flux point ending line l, over the line's points
    {
        std::vector<double> I0((size_t)2 * n);
        for (int e = 0; e < 2; ++e)
            for (int q = 0; q < n; ++q) I0[(size_t)e * n + q] = el.M0[(size_t)fl[e] * nu + pts[0][q]];
        bool ok = true;
        std::vector<double> rec(nu);
        for (int l = 0; l < NLT && ok; ++l)
            for (int e = 0; e < 2 && ok; ++e) {
                std::fill(rec.begin(), rec.end(), 0.0);
                for (int q = 0; q < n; ++q) rec[pts[l][q]] = I0[(size_t)e * n + q];
                ok = close(rec, &el.M0[(size_t)fl[2 * l + e] * nu], nu);
            }
        // every flux point ends exactly one line
        std::vector<int> seen(nf, 0);
        for (int f : fl) seen[f]++;
        for (int f = 0; f < nf && ok; ++f) ok = seen[f] == 1;
        L.interp = ok;
        L.I0 = I0;
    }
    L.n = n;
    L.fl = fl;
    return L;
}

void upload_device(fr_ctx* c) {
    fr::DevCtx& D = c->dev;
    const bool fp64 = c->prm.precision == FR_PREC_FP64;
    const size_t rs = fp64 ? sizeof(double) : sizeof(float);
    const int d = c->ndims, V = c->nvars;
    const bool ns = c->prm.system == FR_NAVIER_STOKES;
    CK(cudaSetDevice(D.device));
    size_t maxpart = 0;
    for (size_t b = 0; b < c->hblocks.size(); ++b) {
        const fr::HostBlock& hb = c->hblocks[b];
        const fr::ElemType& el = *hb.el;
        fr::DevBlock B;
        B.etype = hb.etype; B.nupts = el.nupts; B.nfpts = el.nfpts; B.nvars = V;
        B.nelem = hb.nelem;
        B.ld = round_up(std::max<int64_t>(hb.nelem, 1), 128);
        const int64_t ld = B.ld, nu = el.nupts, nf = el.nfpts;
        maxpart = std::max(maxpart, (size_t)nu * V);
        // metric terms at solution points, filled directly in the compute type
        if (fp64) {
            fill_metrics<double>(c, hb, B, d);
        } else {
            fill_metrics<float>(c, hb, B, d);
        }
        B.Uf = dalloc(c, (size_t)nf * V * ld * rs);
        B.Q = dalloc(c, (size_t)d * nu * V * ld * rs);
        CK(cudaMemset(B.Uf, 0, (size_t)nf * V * ld * rs));
        CK(cudaMemset(B.Q, 0, (size_t)d * nu * V * ld * rs));
        if (ns) {
            B.Qf = dalloc(c, (size_t)d * nf * V * ld * rs);
            CK(cudaMemset(B.Qf, 0, (size_t)d * nf * V * ld * rs));
        }
        B.opM0 = upload_real(c, el.M0, fp64);
        {
            // structured form of M0: the nonzeros of every row, if no row has more than 8
            int nnz = 0;
            const auto nz = nonzero_rows(el.M0, nf, nu, &nnz);
            if (nnz > 0 && nnz <= 8 && fr::interp_prepare((int)nu, (int)nf, nnz, fp64) == cudaSuccess) {
                B.sp_nnz = nnz;
                upload_idx_val(c, nz, nnz, fp64, &B.sp_idx, &B.sp_val);
            }
            (void)cudaGetLastError();
        }
        B.opQ = upload_real(c, hcat(el.M6, (int)nf, el.M46, (int)nu, d * (int)nu), fp64);
        {
            const LineForm lf = line_form(el, d);
            if (lf.n > 0) {
                B.ln_grad = ns && lf.grad && fr::line_prepare(0, d, lf.n, (int)nf, fp64) == cudaSuccess;
                B.ln_div = lf.div && fr::line_prepare(1, d, lf.n, (int)nf, fp64) == cudaSuccess;
                (void)cudaGetLastError();
                if (B.ln_grad || B.ln_div) {
                    B.ln_n = lf.n;
                    std::copy(lf.A.begin(), lf.A.end(), B.ln_A);
                    std::copy(lf.B.begin(), lf.B.end(), B.ln_B);
                    B.ln_fl = (int*)upload(c, lf.fl);
                    B.ln_interp = lf.interp;
                    std::copy(lf.I0.begin(), lf.I0.end(), B.ln_I0);
                }
            }
        }
        {
            // structured form of the divergence operator [M3 | M1 - M3 M2] (same
            // rule): on tensor elements row s holds, per direction, the p+1
            // points of the line through s and the two flux points at its ends
            int nnz = 0;
            const auto nzr = nonzero_rows(hcat(el.M3, (int)nf, el.M132, d * (int)nu, (int)nu), nu, nf + d * nu, &nnz);
            if (nnz > 0 && nnz <= 24 && fr::div_prepare((int)nu, (int)nf, d, nnz, fp64) == cudaSuccess) {
                B.ds_nnz = nnz;
                B.ds_ent = upload_pairs(c, nzr, nnz, fp64);
            }
            (void)cudaGetLastError();
        }
        if (ns) {
            // structured form of the corrected-gradient operator [M6 | M4 - M6 M0]
            // (same rule as M0's): on tensor elements row (i, s) holds the p+1
            // solution points on the line through s in direction i and the two
            // flux points at its ends
            int nnz = 0;
            const auto nzr = nonzero_rows(hcat(el.M6, (int)nf, el.M46, (int)nu, d * (int)nu), d * nu, nf + nu, &nnz);
            if (nnz > 0 && nnz <= 8 && fr::grad_prepare((int)nu, (int)nf, d, nnz, fp64) == cudaSuccess) {
                B.gs_nnz = nnz;
                B.gs_ent = upload_pairs(c, nzr, nnz, fp64);
            }
            (void)cudaGetLastError();
        }
        B.opR = upload_real(c, hcat(el.M3, (int)nf, el.M132, d * (int)nu, (int)nu), fp64);
        {
            // transposed operators of the discrete adjoint
            auto transpose = [](const std::vector<double>& A, int r, int cl) {
                std::vector<double> t((size_t)r * cl);
                for (int i = 0; i < r; ++i)
                    for (int j = 0; j < cl; ++j) t[(size_t)j * r + i] = A[(size_t)i * cl + j];
                return t;
            };
            auto M3T = transpose(el.M3, (int)nu, (int)nf), M132T = transpose(el.M132, (int)nu, d * (int)nu),
                 M0T = transpose(el.M0, (int)nf, (int)nu);
            B.opM3T = upload_real(c, M3T, fp64);
            B.opM132T = upload_real(c, M132T, fp64);
            B.opM0T = upload_real(c, M0T, fp64);
            std::vector<double> M6T, OutT;
            if (ns) {
                // gradient chain: C and U enter Q~ through M6 and M4 - M6 M0
                M6T = transpose(el.M6, d * (int)nu, (int)nf);
                OutT = hcat(M0T, (int)nf, transpose(el.M46, d * (int)nu, (int)nu), d * (int)nu, (int)nu);
                B.opM6T = upload_real(c, M6T, fp64);
                B.opOutT = upload_real(c, OutT, fp64);
            }
            {
                // the same operators in structured form where they allow (tensor
                // elements: p+1 or 2 D nonzeros per row; [M0^T | (M4 - M6 M0)^T]:
                // 2 D + D (p+1))
                const std::vector<double>* ops[6] = {nullptr, &M3T, &M132T, &M0T, ns ? &M6T : nullptr,
                                                     ns ? &OutT : nullptr};
                const int rows[6] = {0, (int)nf, d * (int)nu, (int)nu, (int)nf, (int)nu};
                const int cols[6] = {0, (int)nu, (int)nu, (int)nf, d * (int)nu, (int)(nf + d * nu)};
                for (int w = 1; w < 6; ++w) {
                    if (!ops[w]) continue;
                    int nnz = 0;
                    const auto nz = nonzero_rows(*ops[w], rows[w], cols[w], &nnz);
                    if (w < 5 && fr::sparse_prepare(0, rows[w], cols[w], nnz, fp64)) {
                        B.adj_nnz[w] = nnz;
                        upload_idx_val(c, nz, nnz, fp64, &B.adj_idx[w], &B.adj_val[w]);
                    } else if (w == 5 && fr::sparse_prepare(1, rows[w], cols[w], nnz, fp64)) {
                        B.adj_nnz[5] = nnz;
                        B.adj_ent = upload_pairs(c, nz, nnz, fp64);
                    }
                    (void)cudaGetLastError();
                }
            }
            if (c->prm.precision == FR_PREC_BF16X3 || c->prm.precision == FR_PREC_TF32X3) {
                const int kind = c->prm.precision == FR_PREC_TF32X3 ? 0 : 1;
                B.tcM3T = upload(c, fr::tc::pack_operator(kind, M3T, (int)nf, (int)nu, 0));
                B.tcM132T = upload(c, fr::tc::pack_operator(kind, M132T, d * (int)nu, (int)nu, 0));
                B.tcM0T = upload(c, fr::tc::pack_operator(kind, M0T, (int)nu, (int)nf, 0));
                if (ns) {
                    B.tcM6T = upload(c, fr::tc::pack_operator(kind, M6T, (int)nf, d * (int)nu, 0));
                    B.tcOutT = upload(c, fr::tc::pack_operator(kind, OutT, (int)nu, (int)nf, d * (int)nu));
                }
            }
        }
        if (c->prm.precision == FR_PREC_BF16X3 || c->prm.precision == FR_PREC_TF32X3) {
            const int kind = c->prm.precision == FR_PREC_TF32X3 ? 0 : 1;
            B.tcM0 = upload(c, fr::tc::pack_operator(kind, el.M0, (int)nf, (int)nu, 0));
            // corrected-gradient operator with its rows reordered point-major,
            // (i, s) -> s * d + i, for the fused gradient transform epilogue
            const std::vector<double> Q = hcat(el.M6, (int)nf, el.M46, (int)nu, d * (int)nu);
            const size_t kq = nf + nu;
            std::vector<double> Qp(Q.size());
            for (int i = 0; i < d; ++i)
                for (size_t s = 0; s < nu; ++s)
                    std::copy(&Q[((size_t)i * nu + s) * kq], &Q[((size_t)i * nu + s) * kq] + kq,
                              &Qp[(s * d + i) * kq]);
            B.tcQ = upload(c, fr::tc::pack_operator(kind, Qp, d * (int)nu, (int)nf, (int)nu, d));
            B.tcR = upload(c, fr::tc::pack_operator(kind, hcat(el.M3, (int)nf, el.M132, d * (int)nu, (int)nu),
                                                    (int)nu, (int)nf, (int)(d * nu)));
        }
        if ((double)nf * V * ld >= 4294967296.0) throw Fail{FR_ERR_UNSUPPORTED, "flux-point array exceeds 2^32 entries"};
        D.blocks.push_back(B);
    }
    // interior pair groups by (bL, bR)
    std::map<std::pair<int, int>, std::vector<int64_t>> groups;
    for (int64_t k = 0; k < (int64_t)c->pairs.size(); ++k) groups[{c->pairs[k].bL, c->pairs[k].bR}].push_back(k);
    for (auto& kv : groups) {
        fr::DevPairGroup g;
        g.bL = kv.first.first; g.bR = kv.first.second;
        g.n = (int64_t)kv.second.size();
        const fr::DevBlock &L = D.blocks[g.bL], &R = D.blocks[g.bR];
        std::vector<uint32_t> oL(g.n), oR(g.n);
        std::vector<double> nrm((size_t)d * g.n), mL(g.n), mR(g.n);
        for (int64_t i = 0; i < g.n; ++i) {
            const fr::HostPair& P = c->pairs[kv.second[i]];
            oL[i] = (uint32_t)((int64_t)P.fL * V * L.ld + P.nL);
            oR[i] = (uint32_t)((int64_t)P.fR * V * R.ld + P.nR);
            for (int j = 0; j < d; ++j) nrm[(size_t)j * g.n + i] = P.nrm[j];
            mL[i] = P.magL; mR[i] = P.magR;
        }
        g.offL = (uint32_t*)upload(c, oL);
        g.offR = (uint32_t*)upload(c, oR);
        g.nrm = upload_real(c, nrm, fp64);
        g.magL = upload_real(c, mL, fp64);
        g.magR = upload_real(c, mR, fp64);
        D.pgroups.push_back(g);
    }
    // boundary groups by (block, type)
    std::map<std::pair<int, int>, std::vector<int64_t>> bg;
    for (int64_t k = 0; k < (int64_t)c->bnds.size(); ++k) bg[{c->bnds[k].b, c->bnds[k].bctype}].push_back(k);
    for (auto& kv : bg) {
        fr::DevBndGroup g;
        g.b = kv.first.first; g.bctype = kv.first.second;
        g.n = (int64_t)kv.second.size();
        const fr::DevBlock& B = D.blocks[g.b];
        std::vector<uint32_t> o(g.n);
        std::vector<double> nrm((size_t)d * g.n), m(g.n);
        for (int64_t i = 0; i < g.n; ++i) {
            const fr::HostBnd& P = c->bnds[kv.second[i]];
            o[i] = (uint32_t)((int64_t)P.f * V * B.ld + P.n);
            for (int j = 0; j < d; ++j) nrm[(size_t)j * g.n + i] = P.nrm[j];
            m[i] = P.mag;
        }
        g.off = (uint32_t*)upload(c, o);
        g.nrm = upload_real(c, nrm, fp64);
        g.mag = upload_real(c, m, fp64);
        D.bgroups.push_back(g);
    }
    D.flags = (int*)dalloc(c, 2 * sizeof(int));
    CK(cudaMemset(D.flags, 0, 2 * sizeof(int)));
    D.partial = (double*)dalloc(c, std::max<size_t>(maxpart, 1) * sizeof(double));
    CK(cudaDeviceSynchronize());
}

// Keep the elements of partition `rank` (in increasing global order within
// each block): interior pairs with both sides here stay pairs, pairs with one
// side here become exchange pairs (global L/R orientation kept), boundary
// faces here stay.  Every block must keep at least one element.
void localize(fr_ctx* c, const int32_t* part, int nparts, int rank, std::vector<MpiPair>& mp) {
    const int nb = (int)c->hblocks.size();
    std::vector<int64_t> base(nb + 1, 0);
    for (int b = 0; b < nb; ++b) base[b + 1] = base[b] + c->hblocks[b].nelem;
    for (int64_t i = 0; i < base[nb]; ++i)
        if (part[i] < 0 || part[i] >= nparts) throw Fail{FR_ERR_ARG, "partition index out of range"};
    std::vector<std::vector<int64_t>> g2l(nb);
    const int d = c->ndims;
    for (int b = 0; b < nb; ++b) {
        fr::HostBlock& hb = c->hblocks[b];
        g2l[b].assign(hb.nelem, -1);
        std::vector<double> nodes;
        int64_t k = 0;
        const size_t per = (size_t)hb.nnodes * d;
        for (int64_t e = 0; e < hb.nelem; ++e)
            if (part[base[b] + e] == rank) {
                g2l[b][e] = k++;
                nodes.insert(nodes.end(), hb.nodes.begin() + e * per, hb.nodes.begin() + (e + 1) * per);
            }
        if (k == 0) throw Fail{FR_ERR_ARG, "every element block needs elements in every partition"};
        hb.nodes.swap(nodes);
        hb.nelem = k;
    }
    std::vector<fr::HostPair> keep;
    for (const fr::HostPair& P : c->pairs) {
        const int pL = part[base[P.bL] + P.nL], pR = part[base[P.bR] + P.nR];
        if (pL == rank && pR == rank) {
            fr::HostPair Q = P;
            Q.nL = g2l[P.bL][P.nL];
            Q.nR = g2l[P.bR][P.nR];
            keep.push_back(Q);
        } else if (pL == rank || pR == rank) {
            MpiPair m;
            m.mine_L = pL == rank;
            m.q = m.mine_L ? pR : pL;
            m.b = m.mine_L ? P.bL : P.bR;
            m.f = m.mine_L ? P.fL : P.fR;
            m.n = m.mine_L ? g2l[P.bL][P.nL] : g2l[P.bR][P.nR];
            m.key = {P.bL, P.nL, P.fL};
            for (int j = 0; j < 3; ++j) m.nrm[j] = P.nrm[j];
            m.magL = P.magL;
            m.magR = P.magR;
            mp.push_back(m);
        }
    }
    c->pairs.swap(keep);
    std::vector<fr::HostBnd> bk;
    for (const fr::HostBnd& B : c->bnds)
        if (part[base[B.b] + B.n] == rank) {
            fr::HostBnd C = B;
            C.n = g2l[B.b][B.n];
            bk.push_back(C);
        }
    c->bnds.swap(bk);
    c->part_rank = rank;
    c->part_n = nparts;
}

// Exchange slots and device tables of the partition pairs.  With each
// neighbour q, slots hold first the pairs whose global L side lies on the
// lower of the two ranks, then the others, each sorted by the global L key;
// both ranks derive the same order from the global pairing.
void upload_part(fr_ctx* c, std::vector<MpiPair>& mp) {
    const int rank = c->part_rank, d = c->ndims, V = c->nvars;
    const bool fp64 = c->prm.precision == FR_PREC_FP64;
    const size_t rs = fp64 ? sizeof(double) : sizeof(float);
    const bool ns = c->prm.system == FR_NAVIER_STOKES;
    std::map<int, std::vector<int64_t>> byq;
    for (int64_t k = 0; k < (int64_t)mp.size(); ++k) byq[mp[k].q].push_back(k);
    fr::DevCtx& D = c->dev;
    for (auto& kv : byq) {
        const int q = kv.first;
        std::vector<int64_t>& ids = kv.second;
        const bool lower = rank < q;
        std::stable_sort(ids.begin(), ids.end(), [&](int64_t x, int64_t y) {
            const bool fx = mp[x].mine_L == lower, fy = mp[y].mine_L == lower;   // L side on the lower rank
            if (fx != fy) return fx;
            return mp[x].key < mp[y].key;
        });
        const int nbi = (int)D.nbrs.size();
        fr::DevNeighbour nbr;
        nbr.q = q;
        nbr.nslots = (int64_t)ids.size();
        c->nbr_q.push_back(q);
        c->nbr_keys.emplace_back();
        for (int64_t i : ids) c->nbr_keys.back().push_back(mp[i].key);
        nbr.send_u = dalloc(c, (size_t)V * nbr.nslots * rs);
        nbr.recv_u = dalloc(c, (size_t)V * nbr.nslots * rs);
        // the Q receive buffer also takes the discarded remote-side common solution
        nbr.recv_q = dalloc(c, (size_t)(ns ? d : 1) * V * nbr.nslots * rs);
        nbr.send_q = ns ? dalloc(c, (size_t)d * V * nbr.nslots * rs) : nullptr;
        D.nbrs.push_back(nbr);
        // device groups by (my block, orientation)
        std::map<std::pair<int, int>, std::vector<int64_t>> grp;     // -> slots
        for (int64_t sl = 0; sl < (int64_t)ids.size(); ++sl) grp[{mp[ids[sl]].b, mp[ids[sl]].mine_L ? 1 : 0}].push_back(sl);
        for (auto& gv : grp) {
            fr::DevMpiGroup g;
            g.nb = nbi;
            g.b = gv.first.first;
            g.mine_L = gv.first.second == 1;
            g.n = (int64_t)gv.second.size();
            const fr::DevBlock& B = D.blocks[g.b];
            std::vector<uint32_t> off(g.n), slot(g.n);
            std::vector<double> nrm((size_t)d * g.n), mL(g.n), mR(g.n);
            for (int64_t i = 0; i < g.n; ++i) {
                const MpiPair& m = mp[ids[gv.second[i]]];
                off[i] = (uint32_t)((int64_t)m.f * V * B.ld + m.n);
                slot[i] = (uint32_t)gv.second[i];
                for (int j = 0; j < d; ++j) nrm[(size_t)j * g.n + i] = m.nrm[j];
                mL[i] = m.magL;
                mR[i] = m.magR;
            }
            g.off = (uint32_t*)upload(c, off);
            g.slot = (uint32_t*)upload(c, slot);
            g.nrm = upload_real(c, nrm, fp64);
            g.magL = upload_real(c, mL, fp64);
            g.magR = upload_real(c, mR, fp64);
            D.mgroups.push_back(g);
        }
    }
}

}  // namespace

namespace fr {
DevCtx* ctx_dev(fr_ctx* c) { return c ? &c->dev : nullptr; }
bool ctx_is_part(const fr_ctx* c) { return c && c->part_n > 0; }
void ctx_set_error(fr_ctx* c, const char* msg) {
    if (c) c->err = msg;
}
}  // namespace fr

// ====================================================================== ABI
extern "C" {

int32_t fr_version(void) { return 6; }

fr_status fr_fma_peak(int cuda_device, double* fp32_tflops, double* fp64_tflops) {
    if (!fp32_tflops || !fp64_tflops) return FR_ERR_ARG;
    if (cudaSetDevice(cuda_device) != cudaSuccess) return FR_ERR_CUDA;
    return fr::measure_fma(fp32_tflops, fp64_tflops) == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}

const char* fr_last_error(const fr_ctx* ctx) { return ctx ? ctx->err.c_str() : g_setup_err.c_str(); }

void fr_destroy(fr_ctx* ctx) {
    if (!ctx) return;
    if (ctx->dev.device >= 0) {
        cudaSetDevice(ctx->dev.device);
        cudaDeviceSynchronize();
        fr::prof_free(ctx->dev);
        if (ctx->rk_exec) cudaGraphExecDestroy(ctx->rk_exec);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        if (ctx->xstream) cudaStreamDestroy(ctx->xstream);
        for (cudaEvent_t e : ctx->xev)
            if (e) cudaEventDestroy(e);
        for (void* p : ctx->allocs) cudaFree(p);
    }
    delete ctx;
}

static fr_status setup_impl(const fr_mesh* mesh, const fr_params* prm, int device, const int32_t* part, int nparts,
                            int rank, fr_ctx** out) {
    if (out) *out = nullptr;
    if (!mesh || !prm || !out) return set_err(nullptr, FR_ERR_ARG, "NULL argument");
    if (prm->ndims != 2 && prm->ndims != 3) return set_err(nullptr, FR_ERR_ARG, "ndims must be 2 or 3");
    if (mesh->ndims != prm->ndims) return set_err(nullptr, FR_ERR_ARG, "mesh and params disagree on ndims");
    if (prm->system != FR_EULER && prm->system != FR_NAVIER_STOKES) return set_err(nullptr, FR_ERR_ARG, "bad system");
    if (prm->precision < FR_PREC_FP64 || prm->precision > FR_PREC_TF32X3)
        return set_err(nullptr, FR_ERR_ARG, "bad precision");
    if (mesh->nblocks < 1 || !mesh->blocks) return set_err(nullptr, FR_ERR_ARG, "no element blocks");
    if (mesh->nperiodic < 0 || (mesh->nperiodic > 0 && !mesh->periodic))
        return set_err(nullptr, FR_ERR_ARG, "bad periodic translations");
    if (mesh->nbfaces < 0 || (mesh->nbfaces > 0 && !mesh->bfaces)) return set_err(nullptr, FR_ERR_ARG, "bad boundary list");
    std::unique_ptr<fr_ctx> c(new (std::nothrow) fr_ctx());
    if (!c) return set_err(nullptr, FR_ERR_OOM, "host allocation failed");
    c->prm = *prm;
    c->ndims = prm->ndims;
    c->nvars = prm->ndims + 2;
    try {
        std::map<int, fr::ElemType*> cache;
        int nfp_face = -1;
        for (int b = 0; b < mesh->nblocks; ++b) {
            const fr_eblock& eb = mesh->blocks[b];
            int et = eb.etype;
            if (et < 0 || et > 2) throw Fail{FR_ERR_ARG, "bad element type"};
            if ((et == FR_HEX) != (prm->ndims == 3)) throw Fail{FR_ERR_ARG, "element type does not match ndims"};
            if (eb.nelem < 1 || !eb.nodes) throw Fail{FR_ERR_ARG, "empty element block"};
            if (!cache.count(et)) {
                std::unique_ptr<fr::ElemType> el(new fr::ElemType());
                std::string err;
                if (et == FR_TRI && prm->correction != FR_CORR_DG)
                    throw Fail{FR_ERR_UNSUPPORTED, "SD / HU correction functions are defined for quads and hexes only"};
                if (!fr::build_element(et, prm->order, *el, err, prm->correction)) throw Fail{FR_ERR_ARG, err};
                cache[et] = el.get();
                c->etypes.push_back(std::move(el));
            }
            fr::HostBlock hb;
            hb.etype = et; hb.nnodes = eb.nnodes; hb.nelem = eb.nelem; hb.el = cache[et];
            long double x[3] = {0, 0, 0}, N[27], dN[81];
            if (!fr::shape_functions(et, eb.nnodes, x, N, dN)) throw Fail{FR_ERR_ARG, "unsupported nodes per element"};
            hb.nodes.assign(eb.nodes, eb.nodes + (size_t)eb.nelem * eb.nnodes * prm->ndims);
            if (!fr::prepare_block(hb)) throw Fail{FR_ERR_ARG, "unsupported element mapping"};
            if (nfp_face >= 0 && nfp_face != hb.el->nfp_face) throw Fail{FR_ERR_ARG, "inconsistent face point counts"};
            nfp_face = hb.el->nfp_face;
            c->hblocks.push_back(std::move(hb));
        }
        std::string err;
        if (!fr::pair_mesh(prm->ndims, c->hblocks, mesh->bfaces, mesh->nbfaces, mesh->periodic, mesh->nperiodic,
                           c->pairs, c->bnds, err))
            throw Fail{FR_ERR_MESH, err};
        std::vector<MpiPair> mp;
        if (part) localize(c.get(), part, nparts, rank, mp);
        // locality order: group by block pair, then L flux point, then L element
        std::sort(c->pairs.begin(), c->pairs.end(), [](const fr::HostPair& a, const fr::HostPair& b) {
            if (a.bL != b.bL) return a.bL < b.bL;
            if (a.bR != b.bR) return a.bR < b.bR;
            if (a.fL != b.fL) return a.fL < b.fL;
            return a.nL < b.nL;
        });
        std::sort(c->bnds.begin(), c->bnds.end(), [](const fr::HostBnd& a, const fr::HostBnd& b) {
            if (a.b != b.b) return a.b < b.b;
            if (a.bctype != b.bctype) return a.bctype < b.bctype;
            if (a.f != b.f) return a.f < b.f;
            return a.n < b.n;
        });
        c->dev.ndims = prm->ndims; c->dev.nvars = c->nvars; c->dev.system = prm->system;
        c->dev.precision = prm->precision; c->dev.order = prm->order;
        fr::DevParams& P = c->dev.prm;
        P.gamma = prm->gamma; P.mu = prm->mu; P.prandtl = prm->prandtl; P.beta = prm->ldg_beta; P.tau = prm->ldg_tau;
        if (prm->ref_rho < 0 || (prm->ref_rho == 0 && prm->ref_p != 0))
            throw Fail{FR_ERR_ARG, "perturbation form needs ref_rho > 0 (or ref_rho = ref_p = 0)"};
        P.ref_rho = prm->ref_rho;
        P.ref_p = prm->ref_rho > 0 ? prm->ref_p : 0.0;
        P.ref_E = P.ref_p / (prm->gamma - 1.0);
        P.ref_h = prm->ref_rho > 0 ? prm->gamma * P.ref_E / prm->ref_rho : 0.0;
        P.bc_rho = prm->bc_rho; P.bc_p = prm->bc_p; P.outflow_p = prm->outflow_p; P.wall_cpTw = prm->wall_cpTw;
        for (int i = 0; i < 3; ++i) {
            P.bc_v[i] = prm->bc_v[i];
            P.wall_v[i] = prm->wall_v[i];
            P.wall2_v[i] = prm->wall2_v[i];
        }
        if (device >= 0) {
            c->dev.device = device;
            upload_device(c.get());
            if (part) upload_part(c.get(), mp);
            if (prm->precision == FR_PREC_BF16X3 || prm->precision == FR_PREC_TF32X3) CK(fr::tc::prepare());
            fr::noalloc_prepare(device);
            // the host pair list is only kept for inspection of small meshes
            if (c->pairs.size() > (size_t)4000000) { c->pairs.clear(); c->pairs.shrink_to_fit(); }
        } else {
            if (part) {                   // slot tables for inspection
                c->dev.device = -1;
                std::map<int, std::vector<MpiPair>> byq;
                for (auto& m : mp) byq[m.q].push_back(m);
                for (auto& kv : byq) {
                    const bool lower = rank < kv.first;
                    std::stable_sort(kv.second.begin(), kv.second.end(), [&](const MpiPair& x, const MpiPair& y) {
                        const bool fx = x.mine_L == lower, fy = y.mine_L == lower;
                        if (fx != fy) return fx;
                        return x.key < y.key;
                    });
                    c->nbr_q.push_back(kv.first);
                    c->nbr_keys.emplace_back();
                    for (auto& m : kv.second) c->nbr_keys.back().push_back(m.key);
                }
            }
            // host-only: still check every Jacobian
            for (auto& hb : c->hblocks) {
                std::vector<double> adj((size_t)hb.el->nupts * 9), det(hb.el->nupts);
                for (int64_t e = 0; e < hb.nelem; ++e)
                    if (!fr::element_metrics(hb, e, adj.data(), det.data()))
                        throw Fail{FR_ERR_MESH, "non-positive Jacobian at a solution point"};
            }
        }
    } catch (const Fail& f) {
        if (c->dev.device >= 0)
            for (void* p : c->allocs) cudaFree(p);
        return set_err(nullptr, f.st, f.msg);
    } catch (const std::bad_alloc&) {
        if (c->dev.device >= 0)
            for (void* p : c->allocs) cudaFree(p);
        return set_err(nullptr, FR_ERR_OOM, "host allocation failed");
    }
    *out = c.release();
    return FR_OK;
}

fr_status fr_setup(const fr_mesh* mesh, const fr_params* prm, int device, fr_ctx** out) {
    return setup_impl(mesh, prm, device, nullptr, 0, 0, out);
}

fr_status fr_setup_part(const fr_mesh* mesh, const fr_params* prm, int device, const int32_t* part, int32_t nparts,
                        int32_t rank, fr_ctx** out) {
    if (out) *out = nullptr;
    if (!part || nparts < 1 || rank < 0 || rank >= nparts) return set_err(nullptr, FR_ERR_ARG, "bad partition arguments");
    return setup_impl(mesh, prm, device, part, nparts, rank, out);
}

fr_status fr_part_slots(const fr_ctx* ctx, int32_t* nnbr, int32_t* ranks, int64_t* nslots, int64_t* keys) {
    if (!ctx || !nnbr) return FR_ERR_ARG;
    *nnbr = (int32_t)ctx->nbr_q.size();
    int64_t o = 0;
    for (size_t k = 0; k < ctx->nbr_q.size(); ++k) {
        if (ranks) ranks[k] = ctx->nbr_q[k];
        if (nslots) nslots[k] = (int64_t)ctx->nbr_keys[k].size();
        if (keys)
            for (auto& key : ctx->nbr_keys[k]) {
                keys[3 * o] = key[0]; keys[3 * o + 1] = key[1]; keys[3 * o + 2] = key[2];
                ++o;
            }
    }
    return FR_OK;
}

fr_status fr_layout(const fr_ctx* ctx, int b, int32_t* nupts, int32_t* nfpts, int32_t* nvars, int64_t* nelem,
                    int64_t* ld) {
    if (!ctx || b < 0 || b >= (int)ctx->hblocks.size()) return FR_ERR_ARG;
    const fr::HostBlock& hb = ctx->hblocks[b];
    if (nupts) *nupts = hb.el->nupts;
    if (nfpts) *nfpts = hb.el->nfpts;
    if (nvars) *nvars = ctx->nvars;
    if (nelem) *nelem = hb.nelem;
    if (ld) *ld = round_up(std::max<int64_t>(hb.nelem, 1), 128);
    return FR_OK;
}

fr_status fr_solution_points(const fr_ctx* ctx, int b, double* out) {
    if (!ctx || !out || b < 0 || b >= (int)ctx->hblocks.size()) return FR_ERR_ARG;
    const fr::HostBlock& hb = ctx->hblocks[b];
    const fr::ElemType& el = *hb.el;
    int d = el.ndims, nu = el.nupts, nn = hb.nnodes;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < hb.nelem; ++e)
        for (int s = 0; s < nu; ++s)
            for (int i = 0; i < d; ++i) {
                double acc = 0;
                for (int a = 0; a < nn; ++a) acc += hb.Nu[(size_t)s * nn + a] * hb.nodes[((size_t)e * nn + a) * d + i];
                out[((size_t)i * nu + s) * hb.nelem + e] = acc;
            }
    return FR_OK;
}

fr_status fr_operator(const fr_ctx* ctx, int b, int which, double* out, int32_t* rows, int32_t* cols) {
    if (!ctx || b < 0 || b >= (int)ctx->hblocks.size()) return FR_ERR_ARG;
    const fr::ElemType& el = *ctx->hblocks[b].el;
    int nu = el.nupts, nf = el.nfpts, d = el.ndims, r = 0, cl = 0;
    const std::vector<double>* m = nullptr;
    switch (which) {
        case 0: m = &el.M0; r = nf; cl = nu; break;
        case 1: m = &el.M1; r = nu; cl = d * nu; break;
        case 2: m = &el.M2; r = nf; cl = d * nu; break;
        case 3: m = &el.M3; r = nu; cl = nf; break;
        case 4: m = &el.M4; r = d * nu; cl = nu; break;
        case 6: m = &el.M6; r = d * nu; cl = nf; break;
        case 7: m = &el.M46; r = d * nu; cl = nu; break;
        case 8: m = &el.M132; r = nu; cl = d * nu; break;
        default: return FR_ERR_ARG;
    }
    if (rows) *rows = r;
    if (cols) *cols = cl;
    if (out) std::copy(m->begin(), m->end(), out);
    return FR_OK;
}

fr_status fr_pairs(const fr_ctx* ctx, int64_t* npairs, int64_t* out) {
    if (!ctx || !npairs) return FR_ERR_ARG;
    if (ctx->pairs.empty() && ctx->dev.device >= 0 && !ctx->dev.pgroups.empty()) return FR_ERR_UNSUPPORTED;
    *npairs = (int64_t)ctx->pairs.size();
    if (out)
        for (size_t k = 0; k < ctx->pairs.size(); ++k) {
            const fr::HostPair& P = ctx->pairs[k];
            int64_t* o = out + 6 * k;
            o[0] = P.bL; o[1] = P.fL; o[2] = P.nL; o[3] = P.bR; o[4] = P.fR; o[5] = P.nR;
        }
    return FR_OK;
}

static fr_status check_dev(fr_ctx* ctx) {
    if (!ctx) return FR_ERR_ARG;
    if (ctx->dev.device < 0) return set_err(ctx, FR_ERR_UNSUPPORTED, "host-only context has no device state");
    cudaError_t e = cudaSetDevice(ctx->dev.device);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

static bool ptrs_ok(const fr_ctx* ctx, const void* const* p) {
    if (!p) return false;
    for (size_t b = 0; b < ctx->hblocks.size(); ++b)
        if (!p[b]) return false;
    return true;
}

// a partition's right-hand side needs its neighbours: only fr_rhs_parts runs it
static fr_status whole_mesh(fr_ctx* ctx) {
    if (ctx && ctx->part_n > 0)
        return set_err(ctx, FR_ERR_UNSUPPORTED, "partitioned context: use fr_rhs_parts for its right-hand side");
    return FR_OK;
}

fr_status fr_rhs_parts(fr_ctx* const* parts, int32_t nparts, void* const* const* u, void* const* const* r,
                       void* stream) {
    if (!parts || nparts < 1 || !u || !r) return FR_ERR_ARG;
    for (int p = 0; p < nparts; ++p) {
        fr_ctx* c = parts[p];
        if (!c) return FR_ERR_ARG;
        fr_status s = check_dev(c);
        if (s != FR_OK) return s;
        if (c->part_n != nparts || c->part_rank != p)
            return set_err(c, FR_ERR_ARG, "parts[p] must be the context of rank p of this partition");
        if (c->dev.device != parts[0]->dev.device || c->prm.precision != parts[0]->prm.precision ||
            c->prm.system != parts[0]->prm.system)
            return set_err(c, FR_ERR_ARG, "partitions differ in device, precision or system");
        if (!ptrs_ok(c, u[p]) || !ptrs_ok(c, r[p])) return set_err(c, FR_ERR_ARG, "NULL state pointer");
    }
    fr_ctx* c0 = parts[0];
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!c0->xstream && (e = cudaStreamCreateWithFlags(&c0->xstream, cudaStreamNonBlocking)) != cudaSuccess)
        return set_err(c0, FR_ERR_CUDA, cudaGetErrorString(e));
    for (cudaEvent_t& ev : c0->xev)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return set_err(c0, FR_ERR_CUDA, cudaGetErrorString(e));
    const bool ns = c0->prm.system == FR_NAVIER_STOKES;
    const size_t rs = c0->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    auto phase = [&](int ph) -> cudaError_t {
        for (int p = 0; p < nparts; ++p) {
            cudaError_t er = fr::launch_rhs_phases(parts[p]->dev, u[p], r[p], ph, st);
            if (er != cudaSuccess) return er;
        }
        return cudaSuccess;
    };
    // exchange: rank p's send buffer for q into rank q's receive buffer for p
    // (device-to-device copies on the exchange stream)
    auto exchange = [&](bool qbuf, cudaEvent_t after, cudaEvent_t done) -> cudaError_t {
        cudaError_t er = cudaEventRecord(after, st);
        if (er == cudaSuccess) er = cudaStreamWaitEvent(c0->xstream, after, 0);
        for (int p = 0; p < nparts && er == cudaSuccess; ++p) {
            fr::DevCtx& A = parts[p]->dev;
            for (auto& nb : A.nbrs) {
                fr::DevCtx& B = parts[nb.q]->dev;
                const fr::DevNeighbour* back = nullptr;
                for (auto& x : B.nbrs)
                    if (x.q == p) back = &x;
                if (!back || back->nslots != nb.nslots) return cudaErrorInvalidValue;
                const size_t bytes = (size_t)(qbuf ? A.ndims : 1) * A.nvars * nb.nslots * rs;
                er = cudaMemcpyAsync(qbuf ? back->recv_q : back->recv_u, qbuf ? nb.send_q : nb.send_u, bytes,
                                     cudaMemcpyDeviceToDevice, c0->xstream);
                if (er != cudaSuccess) break;
            }
        }
        if (er == cudaSuccess) er = cudaEventRecord(done, c0->xstream);
        return er;
    };
    // interior-pair work overlaps each exchange (Sec. 3.6: int kernels while the mpi data is in flight)
    if ((e = phase(fr::PH_A)) != cudaSuccess || (e = exchange(false, c0->xev[0], c0->xev[1])) != cudaSuccess)
        return set_err(c0, FR_ERR_CUDA, cudaGetErrorString(e));
    if (ns) {
        if ((e = phase(fr::PH_B1)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c0->xev[1], 0)) != cudaSuccess ||
            (e = phase(fr::PH_B2)) != cudaSuccess || (e = exchange(true, c0->xev[2], c0->xev[3])) != cudaSuccess ||
            (e = phase(fr::PH_C1)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c0->xev[3], 0)) != cudaSuccess ||
            (e = phase(fr::PH_C2)) != cudaSuccess)
            return set_err(c0, FR_ERR_CUDA, cudaGetErrorString(e));
    } else {
        if ((e = phase(fr::PH_C1)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c0->xev[1], 0)) != cudaSuccess ||
            (e = phase(fr::PH_C2)) != cudaSuccess)
            return set_err(c0, FR_ERR_CUDA, cudaGetErrorString(e));
    }
    return FR_OK;
}

fr_status fr_rhs(fr_ctx* ctx, void* const* u, void* const* r, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || !ptrs_ok(ctx, r)) return set_err(ctx, FR_ERR_ARG, "NULL state pointer");
    cudaError_t e = fr::launch_rhs(ctx->dev, u, r, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_rhs_host(fr_ctx* ctx, const void* const* u, void* const* r, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, (void* const*)u) || !ptrs_ok(ctx, r)) return set_err(ctx, FR_ERR_ARG, "NULL state pointer");
    cudaStream_t st = (cudaStream_t)stream;
    size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    std::vector<void*> dv(ctx->dev.blocks.size());
    try {
        for (size_t b = 0; b < ctx->dev.blocks.size(); ++b) {
            fr::DevBlock& B = ctx->dev.blocks[b];
            size_t bytes = (size_t)B.nupts * B.nvars * B.ld * rs;
            if (!B.stage) B.stage = dalloc(ctx, bytes);
            dv[b] = B.stage;
            CK(cudaMemcpyAsync(B.stage, u[b], bytes, cudaMemcpyHostToDevice, st));
        }
        CK(fr::launch_rhs(ctx->dev, dv.data(), dv.data(), st));
        for (size_t b = 0; b < ctx->dev.blocks.size(); ++b) {
            fr::DevBlock& B = ctx->dev.blocks[b];
            size_t bytes = (size_t)B.nupts * B.nvars * B.ld * rs;
            CK(cudaMemcpyAsync(r[b], B.stage, bytes, cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    return FR_OK;
}

fr_status fr_euler(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || nsteps < 0) return set_err(ctx, FR_ERR_ARG, "bad argument");
    const size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    try {
        for (auto& B : ctx->dev.blocks)
            if (!B.rk_tmp) B.rk_tmp = dalloc(ctx, (size_t)B.nupts * B.nvars * B.ld * rs);
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    cudaError_t e = fr::launch_euler(ctx->dev, u, dt, nsteps, (cudaStream_t)stream);
    return e == cudaSuccess ? FR_OK : set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
}

fr_status fr_dopri5(fr_ctx* ctx, void* const* u, double dt, int nsteps, double atol, double rtol, double* err,
                    void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || nsteps < 0) return set_err(ctx, FR_ERR_ARG, "bad argument");
    if (err && !(atol > 0.0 && rtol >= 0.0)) return set_err(ctx, FR_ERR_ARG, "atol must be > 0 and rtol >= 0");
    const size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    try {
        for (auto& B : ctx->dev.blocks) {
            const size_t bytes = (size_t)B.nupts * B.nvars * B.ld * rs;
            if (!B.dp_k) B.dp_k = dalloc(ctx, 7 * bytes);
            if (!B.dp_y) B.dp_y = dalloc(ctx, bytes);
        }
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    cudaError_t e = fr::launch_dopri5(ctx->dev, u, dt, nsteps, atol, rtol, err, (cudaStream_t)stream);
    return e == cudaSuccess ? FR_OK : set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
}

fr_status fr_rk4(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || nsteps < 0) return set_err(ctx, FR_ERR_ARG, "bad argument");
    size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    try {
        for (auto& B : ctx->dev.blocks) {
            size_t bytes = (size_t)B.nupts * B.nvars * B.ld * rs;
            if (!B.rk_acc) B.rk_acc = dalloc(ctx, bytes);
            if (!B.rk_tmp) B.rk_tmp = dalloc(ctx, bytes);
        }
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (ctx->use_graphs && !ctx->dev.prof && nsteps > 0) {
        // one RK4 step captured on a private stream, replayed on the caller's stream
        std::vector<void*> key(u, u + ctx->dev.blocks.size());
        if (!ctx->rk_exec || key != ctx->rk_ptrs || dt != ctx->rk_dt) {
            if (ctx->rk_exec) {
                cudaGraphExecDestroy(ctx->rk_exec);
                ctx->rk_exec = nullptr;
            }
            if (!ctx->cap_stream && (e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
                return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t el = fr::launch_rk4(ctx->dev, u, dt, 1, ctx->cap_stream);
                e = cudaStreamEndCapture(ctx->cap_stream, &g);
                if (e == cudaSuccess) e = el;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->rk_exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ctx->rk_exec = nullptr;
                return set_err(ctx, FR_ERR_CUDA, std::string("RK4 graph capture: ") + cudaGetErrorString(e));
            }
            ctx->rk_ptrs = key;
            ctx->rk_dt = dt;
        }
        for (int i = 0; i < nsteps && e == cudaSuccess; ++i) e = cudaGraphLaunch(ctx->rk_exec, st);
    } else {
        e = fr::launch_rk4(ctx->dev, u, dt, nsteps, st);
    }
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_rk_step(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream) {
    return fr_rk4(ctx, u, dt, nsteps, stream);
}

fr_status fr_rk4_host(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || nsteps < 0) return set_err(ctx, FR_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    std::vector<void*> dv(ctx->dev.blocks.size());
    try {
        for (size_t b = 0; b < ctx->dev.blocks.size(); ++b) {
            fr::DevBlock& B = ctx->dev.blocks[b];
            const size_t bytes = (size_t)B.nupts * B.nvars * B.ld * rs;
            if (!B.stage) B.stage = dalloc(ctx, bytes);
            dv[b] = B.stage;
            CK(cudaMemcpyAsync(B.stage, u[b], bytes, cudaMemcpyHostToDevice, st));
        }
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    // the staging pointers do not change between calls, so the captured RK4 step is reused
    if ((s = fr_rk4(ctx, dv.data(), dt, nsteps, stream)) != FR_OK) return s;
    try {
        for (size_t b = 0; b < ctx->dev.blocks.size(); ++b) {
            fr::DevBlock& B = ctx->dev.blocks[b];
            CK(cudaMemcpyAsync(u[b], B.stage, (size_t)B.nupts * B.nvars * B.ld * rs, cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    return FR_OK;
}

static const char* const kTuneNames[fr::TUNE_N] = {"disu", "tgradu", "gradfpts", "tdivf"};

static void drop_graph(fr_ctx* ctx) {
    if (ctx->rk_exec) {                        // a captured RK4 step holds the old kernel choices
        cudaGraphExecDestroy(ctx->rk_exec);
        ctx->rk_exec = nullptr;
    }
}

fr_status fr_autotune(fr_ctx* ctx, void* const* u, int reps, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || reps < 1) return set_err(ctx, FR_ERR_ARG, "bad argument");
    fr::DevCtx& D = ctx->dev;
    if (D.precision < 2) return FR_OK;                       // CUDA-core paths: nothing to choose
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rs = sizeof(float);
    std::vector<void*> tmp(D.blocks.size(), nullptr);
    const bool prof = D.prof;
    cudaError_t e = cudaSuccess;
    try {
        for (size_t b = 0; b < D.blocks.size(); ++b) {
            fr::DevBlock& B = D.blocks[b];
            const size_t bytes = (size_t)B.nupts * B.nvars * B.ld * rs;
            if (!B.rk_acc) B.rk_acc = dalloc(ctx, bytes);
            if (!B.rk_tmp) B.rk_tmp = dalloc(ctx, bytes);
            CK(cudaMalloc(&tmp[b], bytes));
            CK(cudaMemcpyAsync(tmp[b], u[b], bytes, cudaMemcpyDeviceToDevice, st));
        }
        {
            int64_t l0[fr::K_NKERNELS];
            double t0[fr::K_NKERNELS];
            CK(fr::prof_drain(D, l0, t0));             // records of earlier calls are not this tuning's
        }
        D.prof = true;
        // one product and one block at a time: every candidate runs 1 + reps RK4
        // steps of size 0 on the copy (the state does not change), timed per kernel
        // by the profiler; the other blocks' choices stay fixed, so the difference
        // between candidates is this block's
        const int kid[fr::TUNE_N] = {fr::K_DISU, fr::K_TGRADU, fr::K_GRADFPTS, fr::K_TDIVF};
        // a grouped context launches each product once for all blocks: its blocks
        // share one choice, among the variants that fit every block
        const bool grouped = D.group_blocks && D.blocks.size() > 1 && (int)D.blocks.size() <= fr::tc::group_max();
        for (int slot = 0; slot < fr::TUNE_N; ++slot)
            for (size_t b = 0; b < (grouped ? 1 : D.blocks.size()); ++b) {
                fr::DevBlock& B = D.blocks[b];
                if ((slot == fr::TUNE_DISU || slot == fr::TUNE_GRADFPTS) && D.structured_interp) {
                    // products on the structured kernel have no variants to time
                    bool dense = B.sp_nnz <= 0;
                    if (grouped)
                        for (const auto& B2 : D.blocks) dense = dense || B2.sp_nnz <= 0;
                    if (!dense) continue;
                }
                if (slot == fr::TUNE_TGRADU && D.structured_grad) {
                    auto st_ = [&](const fr::DevBlock& X) { return (D.structured_grad == 1 && X.ln_grad) || X.gs_nnz > 0; };
                    bool dense = !st_(B);
                    if (grouped)
                        for (const auto& B2 : D.blocks) dense = dense || !st_(B2);
                    if (!dense) continue;
                }
                if (slot == fr::TUNE_TDIVF && D.structured_div) {
                    auto st_ = [&](const fr::DevBlock& X) { return (D.structured_div == 1 && X.ln_div) || X.ds_nnz > 0; };
                    bool dense = !st_(B);
                    if (grouped)
                        for (const auto& B2 : D.blocks) dense = dense || !st_(B2);
                    if (!dense) continue;
                }
                int cand[8];
                int nc = fr::tune_candidates(D, B, slot, cand);
                if (grouped) {
                    int k = 0;
                    for (int i = 0; i < nc; ++i) {
                        bool fits = true;
                        for (auto& B2 : D.blocks) {
                            int c2[8];
                            const int n2 = fr::tune_candidates(D, B2, slot, c2);
                            fits = fits && std::find(c2, c2 + n2, cand[i]) != c2 + n2;
                        }
                        if (fits) cand[k++] = cand[i];
                    }
                    nc = k;
                }
                if (nc < 2) continue;
                // two passes over the candidates, each candidate's best time kept: the
                // clock under the power cap drifts over a sweep
                double tbest[8];
                for (int i = 0; i < nc; ++i) tbest[i] = 1e300;
                for (int pass = 0; pass < 2; ++pass)
                    for (int i = 0; i < nc; ++i) {
                        B.tune[slot] = cand[i];
                        if (grouped)
                            for (auto& B2 : D.blocks) B2.tune[slot] = cand[i];
                        CK(fr::launch_rk4(D, tmp.data(), 0.0, 1, st));
                        int64_t l[fr::K_NKERNELS];
                        double t[fr::K_NKERNELS];
                        CK(fr::prof_drain(D, l, t));
                        CK(fr::launch_rk4(D, tmp.data(), 0.0, reps, st));
                        CK(fr::prof_drain(D, l, t));
                        tbest[i] = std::min(tbest[i], t[kid[slot]]);
                    }
                int best = cand[0];
                double best_t = tbest[0];
                for (int i = 1; i < nc; ++i)
                    if (tbest[i] < best_t) {
                        best_t = tbest[i];
                        best = cand[i];
                    }
                B.tune[slot] = best;
                if (grouped)
                    for (auto& B2 : D.blocks) B2.tune[slot] = best;
            }
    } catch (const Fail& f) {
        D.prof = prof;
        for (void* p : tmp)
            if (p) cudaFree(p);
        drop_graph(ctx);
        return set_err(ctx, f.st, f.msg);
    }
    D.prof = prof;
    e = cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    drop_graph(ctx);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_get_tuning(const fr_ctx* ctx, char* buf, int64_t size) {
    if (!ctx || !buf || size < 1) return FR_ERR_ARG;
    std::string out;
    for (size_t b = 0; b < ctx->dev.blocks.size(); ++b) {
        const fr::DevBlock& B = ctx->dev.blocks[b];
        if (b) out += ";";
        out += "b" + std::to_string(b) + ":";
        for (int slot = 0; slot < fr::TUNE_N; ++slot) {
            if (slot) out += ",";
            out += kTuneNames[slot];
            out += "=";
            if (B.tune[slot] < 0) {
                out += "default";
            } else {
                const fr::tc::Variant V = fr::tc::variant_of(slot == fr::TUNE_TGRADU ? ctx->ndims : 0, B.tune[slot]);
                out += std::to_string(V.nt) + "." + std::to_string(V.cw) + "." + std::to_string(V.eg);
            }
        }
    }
    if ((int64_t)out.size() + 1 > size) return FR_ERR_ARG;
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return FR_OK;
}

fr_status fr_set_tuning(fr_ctx* ctx, const char* text) {
    if (!ctx || !text) return FR_ERR_ARG;
    if (ctx->dev.device < 0) return set_err(ctx, FR_ERR_UNSUPPORTED, "host-only context has no device state");
    // parse fully before applying anything
    std::vector<std::array<int, fr::TUNE_N>> want(ctx->dev.blocks.size());
    for (size_t b = 0; b < want.size(); ++b) want[b] = {ctx->dev.blocks[b].tune[0], ctx->dev.blocks[b].tune[1],
                                                        ctx->dev.blocks[b].tune[2], ctx->dev.blocks[b].tune[3]};
    std::string t(text);
    size_t pos = 0;
    while (pos < t.size()) {
        size_t end = t.find(';', pos);
        if (end == std::string::npos) end = t.size();
        const std::string part = t.substr(pos, end - pos);
        pos = end + 1;
        if (part.empty()) continue;
        const size_t colon = part.find(':');
        if (part[0] != 'b' || colon == std::string::npos) return set_err(ctx, FR_ERR_ARG, "tuning: expected b<k>:...");
        const int b = std::atoi(part.substr(1, colon - 1).c_str());
        if (b < 0 || b >= (int)want.size()) return set_err(ctx, FR_ERR_ARG, "tuning: block index out of range");
        size_t q = colon + 1;
        while (q < part.size()) {
            size_t e2 = part.find(',', q);
            if (e2 == std::string::npos) e2 = part.size();
            const std::string kv = part.substr(q, e2 - q);
            q = e2 + 1;
            const size_t eq = kv.find('=');
            if (eq == std::string::npos) return set_err(ctx, FR_ERR_ARG, "tuning: expected name=value");
            int slot = -1;
            for (int k = 0; k < fr::TUNE_N; ++k)
                if (kv.substr(0, eq) == kTuneNames[k]) slot = k;
            if (slot < 0) return set_err(ctx, FR_ERR_ARG, "tuning: unknown product " + kv.substr(0, eq));
            const std::string val = kv.substr(eq + 1);
            if (val == "default") {
                want[b][slot] = -1;
                continue;
            }
            int nt = 0, cw = 0, eg = 0;
            if (std::sscanf(val.c_str(), "%d.%d.%d", &nt, &cw, &eg) != 3)
                return set_err(ctx, FR_ERR_ARG, "tuning: expected nt.cw.eg, got " + val);
            int cand[8];
            const int nc = fr::tune_candidates(ctx->dev, ctx->dev.blocks[b], slot, cand);
            int found = -1;
            for (int i = 0; i < nc; ++i) {
                const fr::tc::Variant V = fr::tc::variant_of(slot == fr::TUNE_TGRADU ? ctx->ndims : 0, cand[i]);
                if (V.nt == nt && V.cw == cw && V.eg == eg) found = cand[i];
            }
            if (found < 0) return set_err(ctx, FR_ERR_ARG, "tuning: variant " + val + " does not fit " + kTuneNames[slot]);
            want[b][slot] = found;
        }
    }
    for (size_t b = 0; b < want.size(); ++b)
        for (int k = 0; k < fr::TUNE_N; ++k) ctx->dev.blocks[b].tune[k] = want[b][k];
    drop_graph(ctx);
    return FR_OK;
}

fr_status fr_set_option(fr_ctx* ctx, const char* name, int64_t value) {
    if (!ctx || !name) return FR_ERR_ARG;
    if (std::string(name) == "graphs") {
        ctx->use_graphs = value != 0;
        return FR_OK;
    }
    if (std::string(name) == "structured_interp") {
        ctx->dev.structured_interp = value != 0;
        drop_graph(ctx);
        return FR_OK;
    }
    if (std::string(name) == "structured_grad") {
        if (value < 0 || value > 2) return set_err(ctx, FR_ERR_ARG, "structured_grad must be 0, 1 or 2");
        ctx->dev.structured_grad = (int)value;
        drop_graph(ctx);
        return FR_OK;
    }
    if (std::string(name) == "structured_div") {
        if (value < 0 || value > 2) return set_err(ctx, FR_ERR_ARG, "structured_div must be 0, 1 or 2");
        ctx->dev.structured_div = (int)value;
        drop_graph(ctx);
        return FR_OK;
    }
    if (std::string(name) == "structured_adjoint") {
        ctx->dev.structured_adjoint = value != 0;
        return FR_OK;
    }
    if (std::string(name) == "group_blocks") {
        ctx->dev.group_blocks = value != 0;
        drop_graph(ctx);
        return FR_OK;
    }
    if (std::string(name) == "tc_wait_limit") {
        if (value < 0) return set_err(ctx, FR_ERR_ARG, "tc_wait_limit must be >= 0");
        ctx->dev.tc_wait_limit = value;
        if (ctx->rk_exec) {                    // a captured RK4 step holds the old limit
            cudaGraphExecDestroy(ctx->rk_exec);
            ctx->rk_exec = nullptr;
        }
        return FR_OK;
    }
    return set_err(ctx, FR_ERR_ARG, std::string("unknown option ") + name);
}

static fr_status adjoint_ready(fr_ctx* ctx) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if ((s = whole_mesh(ctx)) != FR_OK) return s;
    size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    const bool ns = ctx->prm.system == FR_NAVIER_STOKES;
    const size_t d = (size_t)ctx->dev.ndims;
    try {
        for (auto& B : ctx->dev.blocks) {
            if (!B.adj_mu) B.adj_mu = dalloc(ctx, (size_t)B.nupts * B.nvars * B.ld * rs);
            if (!B.adj_uf) B.adj_uf = dalloc(ctx, (size_t)B.nfpts * B.nvars * B.ld * rs);
            if (ns && !B.adj_g) B.adj_g = dalloc(ctx, d * B.nupts * B.nvars * B.ld * rs);
            if (ns && !B.adj_x) B.adj_x = dalloc(ctx, d * B.nupts * B.nvars * B.ld * rs);
            if (!B.rk_acc) B.rk_acc = dalloc(ctx, (size_t)B.nupts * B.nvars * B.ld * rs);
            if (!B.rk_tmp) B.rk_tmp = dalloc(ctx, (size_t)B.nupts * B.nvars * B.ld * rs);
        }
    } catch (const Fail& f) {
        return set_err(ctx, f.st, f.msg);
    }
    return FR_OK;
}

fr_status fr_adjoint_rhs(fr_ctx* ctx, void* const* u, void* const* lambda, void* const* out, void* stream) {
    fr_status s = adjoint_ready(ctx);
    if (s != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || !ptrs_ok(ctx, lambda) || !ptrs_ok(ctx, out))
        return set_err(ctx, FR_ERR_ARG, "NULL state pointer");
    for (size_t b = 0; b < ctx->hblocks.size(); ++b)
        if (out[b] == u[b] || out[b] == lambda[b]) return set_err(ctx, FR_ERR_ARG, "out may not alias u or lambda");
    cudaError_t e = fr::launch_adjoint_rhs(ctx->dev, u, lambda, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_rk4_adjoint(fr_ctx* ctx, void* const* u0, void* const* lambda, double dt, int nsteps, int every,
                         void* stream) {
    fr_status s = adjoint_ready(ctx);
    if (s != FR_OK) return s;
    if (!ptrs_ok(ctx, u0) || !ptrs_ok(ctx, lambda) || nsteps < 1 || every < 1)
        return set_err(ctx, FR_ERR_ARG, "bad argument");
    const size_t nb = ctx->dev.blocks.size();
    const size_t rs = ctx->prm.precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    const int nck = (nsteps + every - 1) / every, nblk = std::min(every, nsteps);
    std::vector<void*> mine;
    auto slots = [&](int n) {
        std::vector<std::vector<void*>> v((size_t)n, std::vector<void*>(nb));
        for (int i = 0; i < n; ++i)
            for (size_t b = 0; b < nb; ++b) {
                const fr::DevBlock& B = ctx->dev.blocks[b];
                void* p = nullptr;
                if (cudaMalloc(&p, (size_t)B.nupts * B.nvars * B.ld * rs) != cudaSuccess)
                    throw Fail{FR_ERR_OOM, "checkpoint allocation failed"};
                mine.push_back(p);
                v[(size_t)i][b] = p;
            }
        return v;
    };
    cudaError_t e = cudaSuccess;
    try {
        auto ck = slots(nck), blk = slots(nblk), tmp = slots(8);
        e = fr::launch_rk4_adjoint(ctx->dev, u0, lambda, dt, nsteps, every, ck, blk, tmp, (cudaStream_t)stream);
        cudaError_t e2 = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess) e = e2;
    } catch (const Fail& f) {
        for (void* p : mine) cudaFree(p);
        return set_err(ctx, f.st, f.msg);
    }
    for (void* p : mine) cudaFree(p);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_sum_weighted(fr_ctx* ctx, void* const* u, double* out, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if (!ptrs_ok(ctx, u) || !out) return set_err(ctx, FR_ERR_ARG, "bad argument");
    cudaError_t e = fr::launch_sum_weighted(ctx->dev, u, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_check_finite(fr_ctx* ctx, void* const* u, void* stream) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    if (!ptrs_ok(ctx, u)) return set_err(ctx, FR_ERR_ARG, "NULL state pointer");
    cudaError_t e = fr::launch_check_finite(ctx->dev, u, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_profile_enable(fr_ctx* ctx, int enable) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    ctx->dev.prof = enable != 0;
    return FR_OK;
}

fr_status fr_profile_read(fr_ctx* ctx, int32_t* nk, char* names, int64_t* launches, double* ms) {
    if (!nk) return FR_ERR_ARG;
    *nk = fr::K_NKERNELS;
    if (!names && !launches && !ms) return FR_OK;   // size query only: records are kept
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    int64_t l[fr::K_NKERNELS];
    double t[fr::K_NKERNELS];
    cudaError_t e = fr::prof_drain(ctx->dev, l, t);
    for (int k = 0; k < fr::K_NKERNELS; ++k) {
        if (names) {
            std::memset(names + 32 * k, 0, 32);
            std::strncpy(names + 32 * k, fr::kKernelNames[k], 31);
        }
        if (launches) launches[k] = l[k];
        if (ms) ms[k] = t[k];
    }
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}

fr_status fr_sync_status(fr_ctx* ctx) {
    fr_status s = check_dev(ctx);
    if (s != FR_OK) return s;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    int f[2] = {0, 0};
    e = cudaMemcpy(f, ctx->dev.flags, sizeof(f), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    cudaMemset(ctx->dev.flags, 0, sizeof(f));
    if (f[1]) return set_err(ctx, FR_ERR_TIMEOUT, "a bounded device wait gave up");
    if (f[0]) return set_err(ctx, FR_ERR_NONFINITE, "non-finite value in a state");
    return FR_OK;
}

}  // extern "C"
