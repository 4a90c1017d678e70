// Split-precision tensor-core operator GEMMs (tcgen05), see fr_tc.cu.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace fr {
namespace tc {

// reference state of the perturbation form, subtracted per variable from the
// B rows that hold solution states
struct SubRef {
    float v[5];
};

// Pack an M x (K1 + K2) row-major FP64 operator into the shared-memory operand
// layout of the kernel, split into hi / lo parts: K chunks of segment 1
// (columns [0, K1)) then of segment 2 (columns [K1, K1 + K2)), each padded
// with zero columns to whole chunks.  kind 0 = TF32, 1 = BF16.
// group = g > 1: the rows are (point, component) pairs ordered point-major,
// g per point, and every row block holds whole points (the layout the
// gradient transform epilogue needs).
std::vector<uint8_t> pack_operator(int kind, const std::vector<double>& A, int M, int K1, int K2, int group = 1);

// Gradient transform fused into the epilogue of the corrected-gradient
// product: the operator's rows are s * ndims + i (packed with group ndims),
// and row j * nupts + s of C receives rcp(s) sum_i smat[i][j](s) acc(s, i),
// Q = J^-T Q~ (smat = J J^-1 as [ndims*ndims][nupts][ld], rcp = 1/J as
// [nupts][ld]).  nvars: variables in the N = nvars * ld columns.
struct GradXform {
    const float* smat;
    int ndims, nupts, nvars;
};

// One-time launch set-up (shared-memory limits, SM count) on the current
// device; called at context set-up so that later launches can be captured.
cudaError_t prepare();

// C[M x N] = A [B1; B2]: B1 holds K1 rows, B2 (may be NULL when K2 = 0) K2
// rows, both with row stride N (a multiple of 128).  epi = 1 multiplies row
// r, column c by -rcp[r][c % ld] (-1/J).  Rows of segment `subseg` (1 or 2;
// 0 = none) have sub.v[c / ld] subtracted (perturbation form).  flags[1] is
// raised if a wait gives up.  gx (optional) selects the gradient transform
// epilogue, with rcp = 1/J; rk (optional, epi = 1 semantics) the RK stage
// epilogue (C unused).  Host-side tensor-map encoding failures and
// inconsistent arguments return cudaErrorInvalidValue.
// RK stage fused into the -1/J epilogue: with k = -acc / J (never stored),
// mode 0: acc = u + a k, tmp = u + b k; mode 1: acc += a k, tmp = u + b k;
// mode 2: u = acc + a k.  u, acc, tmp have the layout of C; only columns
// c with c % ld < nelem (real elements) are written.
struct RkFuse {
    int mode;
    float a, b;
    float *u, *acc, *tmp;
    int64_t nelem;
};

// wait_limit: SM clock cycles after which a bounded wait gives up and sets
// flags[1] (0: about two seconds).  variant: index of the kernel variant
// (see variants(); -1: the default rule), cudaErrorInvalidValue if it does
// not fit the operator.
cudaError_t gemm(int kind, int M, int K1, int K2, const void* Apack, const float* B1, const float* B2, int64_t N,
                 float* C, int epi, const float* rcp, int64_t ld, int subseg, SubRef sub, int* flags,
                 cudaStream_t st, const GradXform* gx = nullptr, const RkFuse* rk = nullptr,
                 long long wait_limit = 0, int variant = -1);

// One problem of a grouped launch: C[M x N] = A [B1; B2] with the arguments
// of gemm() (epi and the variant are the group's).
struct GemmProblem {
    int M, K1, K2;
    const void* Apack;
    const float *B1, *B2;
    int64_t N;
    float* C;
    const float* rcp;
    int64_t ld;
    int subseg;
    const GradXform* gx;
    const RkFuse* rk;
};
// The same operator product of up to group_max() element blocks in one
// persistent launch (one work list; all with or all without gx, all with or
// all without rk, gx of one dimension).  The variant must fit every problem.
cudaError_t gemm_group(int kind, int epi, const GemmProblem* probs, int n, SubRef sub, int* flags, cudaStream_t st,
                       long long wait_limit = 0, int variant = -1);
int group_max();

// A kernel variant: 128-column subtiles per work item (1 or 2), converter
// warps and epilogue warp groups.
struct Variant {
    int nt, cw, eg;
};
// Variants that fit an operator of nrp padded rows per row block, for the
// plain / -1/J / RK-stage epilogue (gd = 0) or the gradient transform of gd
// dimensions: their indices into out[] (at most 8); returns the count.
int variants(int gd, int nrp, int* out);
Variant variant_of(int gd, int v);
// padded rows per row block of an M-row operator (group g: whole points of g rows)
int padded_rows(int M, int group);

// whether an M-row operator runs with two 128-column subtiles, the kernels
// that carry the fused RK stage epilogue (M <= 128)
bool rk_fusable(int M);

}  // namespace tc
}  // namespace fr
