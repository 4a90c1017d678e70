// Split-precision operator GEMMs on the 5th-generation tensor cores (tcgen05).
//
// C[M x N] = A[M x K] [B1; B2]  (App. A: every operator product of the FR step
// is such a product with a small constant A and a state matrix B of
// nvars*ld columns).  A and B are FP32 values split into two parts,
// x = x_hi + x_lo, in the MMA input type (TF32: 11+11 significant bits;
// BF16: 8+8), and three products are accumulated in FP32 in tensor memory:
//     C = A_hi B_hi + A_hi B_lo + A_lo B_hi.
// The operator is split once on the host and stored in the shared-memory
// operand layout; the state is split on the fly.
//
// Persistent, warp-specialised kernel (one CTA per SM).  The MMA M dimension
// is 128 state columns (one per TMEM lane) and the N dimension is a block of
// at most 256 operator rows (padded to 16), so each thread of the epilogue
// owns one state column and every row of the block, and each warp store
// writes 32 consecutive columns.  Operators of more than 256 rows are cut into
// equal row blocks; a work item is (column tile, row block), and the row
// blocks of one column tile run on neighbouring CTAs at the same time, so the
// second read of the state tile is served by L2.  Operators of at most 128
// rows take two 128-column subtiles per work item, so that each operator
// chunk feeds two MMAs.
//   warp 0      producer: per K chunk, one bulk copy of the packed operator
//               and one 2D TMA load of the FP32 state tile [chunk rows x
//               128 or 256 columns]; both complete on the stage's "full"
//               mbarrier;
//   warp 1      MMA issuer (one thread) and owner of tensor memory: three
//               tcgen05.mma per 32-byte K step and subtile (state_hi op_hi,
//               state_lo op_hi, state_hi op_lo), committed to the stage's
//               "empty" barrier and, after the last chunk of a work item, to
//               its accumulator barrier;
//   next 4 or 8 warps
//               converters: read the FP32 tile, subtract the perturbation
//               reference where the rows are solution states, split into
//               hi / lo and write the K-major core-matrix operand layout;
//   the rest    epilogue: tcgen05.ld of the accumulators (TMEM lane quadrant
//               = warp % 4; 12 warps interleave 16-row groups when the tile
//               has one subtile, 8 when it has two), optional -1/J
//               scaling or the fused RK stage, coalesced stores.  Direct global stores from four
//               warps could not drain a 160-row accumulator as fast as the
//               MMAs fill the next one; twelve warps keep more stores in
//               flight.
// Shared-memory stages form a ring; accumulators are double-buffered in
// tensor memory whenever two fit.  Every mbarrier wait gives up after a
// cycle limit (about two seconds unless the caller sets a shorter one) and
// raises the context's timeout flag; a CTA then still waits, with its own
// ~2 s limit, for the bulk copies it armed and the MMAs it issued to finish
// before it frees tensor memory and exits.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "fr_dev.hpp"
#include "fr_tc.hpp"

namespace fr {
namespace tc {

constexpr int BN = 128;                        // state columns per subtile (MMA M, one per TMEM lane)
constexpr int KSTEPS = 2;                      // 32-byte MMA K steps per chunk
constexpr int ROWB = 32 * KSTEPS;              // bytes of K per operand row per chunk
constexpr int SPART = BN * ROWB;               // one part (hi or lo) of the state operand per chunk
constexpr int MAX_NST = 6;
constexpr int MAX_RB = 256;                    // operator rows per block (MMA N limit)
constexpr long long DRAIN_LIMIT = 4000000000LL;  // cycles (~2 s) for the end-of-kernel drains, whatever a.limit is

// Byte offset of (row r, K byte kb) inside one operand part: core matrices of
// 8 rows x 16 bytes, 2*KSTEPS of them along K, then the next 8-row group.
__host__ __device__ constexpr int core_off(int r, int kb) {
    return ((r >> 3) * (2 * KSTEPS) + (kb >> 4)) * 128 + (r & 7) * 16 + (kb & 15);
}

// Row blocks of an M-row operator.  group = 1: nrb equal blocks of rr rows
// (a multiple of 16, at most MAX_RB), the last one possibly shorter.  group =
// g > 1 (rows ordered point-major, g rows per point): every block holds whole
// points, rr = g * (points per block), and the MMA width nrp covers whole
// 16-point units, 16 g ceil(points / 16) <= MAX_RB.
struct RowBlocks {
    int nrb, rr, nrp;
};
__host__ __device__ inline RowBlocks row_blocks(int M, int group) {
    RowBlocks r;
    if (group <= 1) {
        const int n0 = (M + MAX_RB - 1) / MAX_RB;
        r.nrp = ((M + n0 - 1) / n0 + 15) / 16 * 16;
        r.rr = r.nrp;
    } else {
        const int npts = M / group, cap = (MAX_RB / (16 * group)) * 16;
        const int n0 = (npts + cap - 1) / cap, ppb = (npts + n0 - 1) / n0;
        r.rr = ppb * group;
        r.nrp = 16 * group * ((ppb + 15) / 16);
    }
    r.nrb = (M + r.rr - 1) / r.rr;              // no empty trailing block
    return r;
}

// 128-column subtiles per work item: two when the row block is at most 128
// rows, so that both accumulators still fit twice in tensor memory
__host__ __device__ constexpr int subtiles_for(int nrp) { return nrp <= 128 ? 2 : 1; }
// Threads of a kernel variant: producer and MMA warps, cw converter warps
// (sets of 4, one warp per scheduler each; the sets split each chunk's
// conversion) and eg epilogue warp groups (4 warps each, one per TMEM lane
// quadrant).
__host__ __device__ constexpr int nthreads_for(int cw, int eg) { return 64 + 32 * cw + 128 * eg; }

struct Layout {
    int nrp;                      // rows per block (MMA N)
    int opart, a_bytes, stg_bytes, off_stg, off_bhi, off_blo, stage, nst, tbuf, smem;
};

__host__ __device__ inline Layout make_layout(int kind, int nrp, int nt) {
    Layout L;
    L.nrp = nrp;
    L.opart = L.nrp * ROWB;
    L.a_bytes = 2 * L.opart;
    const int kce = ROWB / (kind == 0 ? 4 : 2);
    L.stg_bytes = kce * BN * nt * 4;
    L.off_stg = L.a_bytes;
    L.off_bhi = L.off_stg + L.stg_bytes;              // subtile t at + t * SPART
    L.off_blo = L.off_bhi + nt * SPART;
    L.stage = L.off_blo + nt * SPART;
    L.nst = (220 * 1024) / L.stage;
    if (L.nst > MAX_NST) L.nst = MAX_NST;
    L.tbuf = 2 * nt * L.nrp <= 512 ? 2 : 1;
    L.smem = L.nst * L.stage + 1024;
    return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    constexpr uint32_t LBO = 128;                  // next core matrix along K
    constexpr uint32_t SBO = 2 * KSTEPS * 128;     // next 8-row group
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
    return d;
}

template <int KIND>
__device__ __forceinline__ uint32_t instr_desc(int n) {
    // D = F32 (bits 4-5), A/B type (bits 7-9 / 10-12): TF32 = 2 (kind::tf32), BF16 = 1 (kind::f16),
    // both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128 state columns)
    return (1u << 4) | ((KIND == 0 ? 2u : 1u) << 7) | ((KIND == 0 ? 2u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(BN >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long limit) {
    long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint16_t to_bf16(float x) {
    uint32_t u = __float_as_uint(x);
    u += 0x7FFFu + ((u >> 16) & 1u);                // round to nearest even
    return (uint16_t)(u >> 16);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    if (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

struct TcArgs {
    int M;              // operator rows
    int nrb, rr, nrp;   // row blocks, operator rows per block, padded rows per block (MMA N)
    int nch1, nch2;     // K chunks of segment 1 (B1) and 2 (B2)
    int subseg;         // segment whose rows get the reference subtracted (0: none)
    const uint8_t* Apack;   // packed operator: nrb blocks of nch chunks of Layout::a_bytes
    int64_t N, ld;
    float* C;
    int epi;
    const float* rcp;
    float sub0, sub1, sub2, sub3, sub4;
    int* flags;
    long long limit;
    int ntiles;         // column tiles (NT * 128 columns each)
    int nwork;          // ntiles * nrb
    // gradient transform epilogue (epi = 2): rows are (point, direction) pairs
    // s * gD + i; row j * gnu + s of C receives rcp(s) sum_i smat[i][j](s) acc(s, i)
    const float* smat;
    int gD, gnu;
    int vinter;         // > 0: work order interleaves the vinter variables of one element range
    // RK stage epilogue (epi = 3): k = -acc / J, then by rk_mode
    //   0: rk_acc = u + rk_a k, rk_tmp = u + rk_b k;  1: rk_acc += rk_a k, rk_tmp = u + rk_b k;
    //   2: u = rk_acc + rk_a k; only columns of real elements (col % ld < rk_nelem) are written
    int rk_mode;
    float rk_a, rk_b;
    float *rk_u, *rk_acc, *rk_tmp;
    int64_t rk_nelem;
};

// column tile of the tl-th tile in work order
__device__ __forceinline__ int col_tile(const TcArgs& a, int tl) {
    if (!a.vinter) return tl;
    const int per = a.ntiles / a.vinter;
    return (tl % a.vinter) * per + tl / a.vinter;
}

// One launch serves a group of problems (the same operator product of every
// element block of a mixed mesh): their work items form one list, problem
// after problem.  Shared-memory stages and tensor-memory buffers are laid out
// for the group's largest operator block (nrp); each work item's MMA width,
// operator copy and epilogue follow its own problem.
constexpr int MAXG = 4;
struct TcGroup {
    CUtensorMap m[2 * MAXG];      // state tensor maps (segments 1 and 2) of every problem
    TcArgs p[MAXG];
    int ng;
    int wstart[MAXG + 1];         // first work item of each problem; wstart[ng] = all work items
    int nrp;                      // largest padded rows per block of the group
};

__device__ __forceinline__ int group_of(const TcGroup& G, int w) {
    int g = 0;
    while (g + 1 < G.ng && w >= G.wstart[g + 1]) ++g;
    return g;
}

// Epilogue of the gradient transform: 4-point units of one row block,
// q_i = acc(s, i) from tensor memory, Q_j(s) = rcp(s) sum_i adj_ij(s) q_i
// (Q = J^-T Q~, with adj = J J^-1 and rcp = 1/J stored per point).
template <int D>
__device__ __forceinline__ void epi_grad(const TcArgs& a, uint32_t tcol, int p0, int np, int u_first, int u_step,
                                         int64_t col, bool col_ok) {
    const int64_t n = col % a.ld, ld = a.ld, N = a.N;
    const float* sm = a.smat + n;
    const float* rc = a.rcp + n;
    float* cc = a.C + col;
    const int64_t es = (int64_t)a.gnu * ld;           // stride between the D*D metric entries
#pragma unroll 1
    for (int u0 = u_first; u0 < np; u0 += u_step) {
        uint32_t r[4 * D];
        __syncwarp();                                  // reconverge after the lane-dependent stores
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const uint32_t ta = tcol + (uint32_t)(u0 * D + 4 * k);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r[4 * k + 0]), "=r"(r[4 * k + 1]), "=r"(r[4 * k + 2]), "=r"(r[4 * k + 3])
                         : "r"(ta));
        }
        // the metric terms of the unit's 4 points are loaded while the tensor-memory load is in flight
        float m[4][D * D], rj[4];
        if (col_ok) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int s = min(p0 + u0 + k, p0 + np - 1);          // clamped: rows past np are not stored
                const float* ps = sm + (int64_t)s * ld;
#pragma unroll
                for (int e = 0; e < D * D; ++e) m[k][e] = __ldg(ps + e * es);
                rj[k] = __ldg(rc + (int64_t)s * ld);
            }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!col_ok) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = p0 + u0 + k;
            if (u0 + k < np) {
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float acc = 0.f;
#pragma unroll
                    for (int i = 0; i < D; ++i) acc += m[k][i * D + j] * __uint_as_float(r[k * D + i]);
                    cc[((int64_t)j * a.gnu + s) * N] = acc * rj[k];
                }
            }
        }
    }
}

__device__ __forceinline__ float sub_of(const TcArgs& a, int64_t v) {
    return v == 0 ? a.sub0 : v == 1 ? a.sub1 : v == 2 ? a.sub2 : v == 3 ? a.sub3 : a.sub4;
}

// MULTI: the launch serves several problems (found per work item); a
// single-problem launch reads its arguments at fixed parameter offsets
template <int KIND, int NT, int GD, int CONVW, int EG, bool MULTI>
__global__ void __launch_bounds__(nthreads_for(CONVW, EG), 1)
tc_gemm_kernel(const __grid_constant__ TcGroup G) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[MAX_NST], bar_conv[MAX_NST], bar_empty[MAX_NST];
    __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t tmem_holder;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwork = G.wstart[G.ng];
    int* const flags = G.p[0].flags;
    const long long limit = G.p[0].limit;
    const Layout L = make_layout(KIND, G.nrp, NT);
    constexpr int ESZ = KIND == 0 ? 4 : 2;
    constexpr int KCE = ROWB / ESZ;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < L.nst; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_conv[s])), "r"(32 * CONVW));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[s])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_tfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_tempty[b])), "r"(128 * EG));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_drain)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    bool ok = true;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;
            for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
                const int g = (MULTI ? group_of(G, w) : 0);
                const TcArgs& a = G.p[g];
                const int lw = w - G.wstart[g], nch = a.nch1 + a.nch2;
                const int tl = lw / a.nrb, rb = lw - tl * a.nrb;
                const int col0 = col_tile(a, tl) * NT * BN;
                const int ab = 2 * a.nrp * ROWB;                     // this problem's operator chunk
                const uint8_t* ablk = a.Apack + (size_t)rb * nch * ab;
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % L.nst, k = it / L.nst;
                    if (k > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (k - 1) & 1, limit)) { ok = false; break; }
                    uint8_t* st = smem + s * L.stage;
                    const uint32_t fb = smem_u32(&bar_full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"((uint32_t)(ab + L.stg_bytes))
                                 : "memory");
                    const uint8_t* src = ablk + (size_t)c * ab;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(st)),
                        "l"(src), "r"((uint32_t)ab), "r"(fb)
                        : "memory");
                    const bool seg1 = c < a.nch1;
                    const int row0 = (seg1 ? c : c - a.nch1) * KCE;
                    const CUtensorMap* tm = &G.m[2 * g + (seg1 ? 0 : 1)];
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
                        "{%2, %3}], [%4];" ::"r"(smem_u32(st + L.off_stg)),
                        "l"(tm), "r"(col0), "r"(row0), "r"(fb)
                        : "memory");
                }
            }
            // copies possibly still in flight (after any role gave up): wait for the
            // last chunk armed on every stage before the CTA may exit
            for (int i = it > L.nst ? it - L.nst : 0; i < it; ++i)
                if (!mbar_wait(smem_u32(&bar_full[i % L.nst]), (i / L.nst) & 1, DRAIN_LIMIT)) ok = false;
            if (!ok) atomicOr(&flags[1], 1);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int it = 0, wc = 0;
            for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++wc) {
                const TcArgs& a = G.p[(MULTI ? group_of(G, w) : 0)];
                const int nch = a.nch1 + a.nch2;
                const uint32_t id = instr_desc<KIND>(a.nrp);
                const int b = wc % L.tbuf;
                if (!mbar_wait(smem_u32(&bar_tempty[b]), ((wc / L.tbuf) & 1) ^ 1, limit)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dbase = tmem + (uint32_t)(b * NT * L.nrp);
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % L.nst, k = it / L.nst;
                    if (!mbar_wait(smem_u32(&bar_conv[s]), k & 1, limit)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = smem_u32(smem + s * L.stage);
                    const uint32_t o_hi = st, o_lo = st + (uint32_t)(a.nrp * ROWB);   // operator parts (MMA B)
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const uint32_t s_hi = st + L.off_bhi + t * SPART, s_lo = st + L.off_blo + t * SPART;
                        const uint32_t d = dbase + (uint32_t)(t * L.nrp);
#pragma unroll
                        for (int j = 0; j < KSTEPS; ++j) {
                            const uint32_t o = 2 * j * 128;
                            const uint32_t first = (c == 0 && j == 0) ? 0u : 1u;
                            mma<KIND>(d, make_desc(s_hi + o), make_desc(o_hi + o), id, first);
                            mma<KIND>(d, make_desc(s_lo + o), make_desc(o_hi + o), id, 1u);
                            mma<KIND>(d, make_desc(s_hi + o), make_desc(o_lo + o), id, 1u);
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_u32(&bar_empty[s]))
                        : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&bar_tfull[b]))
                             : "memory");
            }
            // MMAs possibly still in flight: one more commit, waited for, before
            // tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar_drain))
                         : "memory");
            if (!mbar_wait(smem_u32(&bar_drain), 0, DRAIN_LIMIT)) ok = false;
            if (!ok) atomicOr(&flags[1], 1);
        }
    } else if (warp < 2 + CONVW) {
        // ---------------------------------------------------------- converters
        // CONVW / 4 sets of 128 threads share each chunk's (subtile, 16-byte K group) pieces
        const int ct = (tid - 64) & 127;               // state column within a subtile = MMA A row
        const int cset = (tid - 64) >> 7;
        constexpr int ncols = NT * BN;
        int it = 0;
        for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
            const int g = (MULTI ? group_of(G, w) : 0);
            const TcArgs& a = G.p[g];
            const int nch = a.nch1 + a.nch2;
            const int tile = col_tile(a, (w - G.wstart[g]) / a.nrb);
            float subv[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int64_t gc = (int64_t)tile * ncols + t * BN + ct;
                subv[t] = gc < a.N ? sub_of(a, gc / a.ld) : 0.f;
            }
            for (int c = 0; c < nch; ++c, ++it) {
                const int s = it % L.nst, k = it / L.nst;
                if (!mbar_wait(smem_u32(&bar_full[s]), k & 1, limit)) { ok = false; break; }
                uint8_t* st = smem + s * L.stage;
                const float* stg = (const float*)(st + L.off_stg);
                const bool seg1 = c < a.nch1;
                const bool dosub = a.subseg == (seg1 ? 1 : 2);
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const float sv = dosub ? subv[t] : 0.f;
                    const int cc = t * BN + ct;
#pragma unroll
                    for (int g = 0; g < ROWB / 16; ++g) {
                        if ((t * (ROWB / 16) + g) % (CONVW / 4) != cset) continue;
                        constexpr int PER = 16 / ESZ;
                        float x[PER];
#pragma unroll
                        for (int q = 0; q < PER; ++q) x[q] = stg[(g * PER + q) * ncols + cc] - sv;
                        uint4 h, l;
                        if (KIND == 0) {
                            uint32_t hh[4], ll[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                hh[q] = to_tf32(x[q]);
                                ll[q] = to_tf32(x[q] - __uint_as_float(hh[q]));
                            }
                            h = make_uint4(hh[0], hh[1], hh[2], hh[3]);
                            l = make_uint4(ll[0], ll[1], ll[2], ll[3]);
                        } else {
                            uint32_t hh[4], ll[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                uint16_t h0 = to_bf16(x[2 * q]), h1 = to_bf16(x[2 * q + 1]);
                                float r0 = x[2 * q] - __uint_as_float((uint32_t)h0 << 16);
                                float r1 = x[2 * q + 1] - __uint_as_float((uint32_t)h1 << 16);
                                hh[q] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                                ll[q] = (uint32_t)to_bf16(r0) | ((uint32_t)to_bf16(r1) << 16);
                            }
                            h = make_uint4(hh[0], hh[1], hh[2], hh[3]);
                            l = make_uint4(ll[0], ll[1], ll[2], ll[3]);
                        }
                        *(uint4*)(st + L.off_bhi + t * SPART + core_off(ct, 16 * g)) = h;
                        *(uint4*)(st + L.off_blo + t * SPART + core_off(ct, 16 * g)) = l;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&bar_conv[s]));
            }
        }
        if (!ok && tid == 64) atomicOr(&flags[1], 1);
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                        // TMEM lane quadrant of this warp
        const int grp = (warp - 2 - CONVW) >> 2;       // 16-row groups grp, grp + EG, ...
        int wc = 0;
        for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++wc) {
            const int g = (MULTI ? group_of(G, w) : 0);
            const TcArgs& a = G.p[g];
            const int lw = w - G.wstart[g];
            const int tl = lw / a.nrb, rb = lw - tl * a.nrb;
            const int tile = col_tile(a, tl);
            const int rbase = rb * a.rr;                          // first operator row of the block
            const int mr = min(a.rr, a.M - rbase);                // real rows in the block
            const int b = wc % L.tbuf;
            // the give-up decision is taken by the whole warp: the tensor-memory loads
            // below are .sync.aligned and must be executed by all 32 lanes or none
            const bool got = mbar_wait(smem_u32(&bar_tfull[b]), (wc / L.tbuf) & 1, limit);
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int64_t col = (int64_t)tile * NT * BN + t * BN + q * 32 + lane;    // this thread's state column
                const bool col_ok = col < a.N && (a.epi != 3 || col % a.ld < a.rk_nelem);
                const uint32_t tcol = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NT * L.nrp + t * L.nrp);
                if constexpr (GD > 0) {
                    epi_grad<GD>(a, tcol, rbase / GD, mr / GD, 4 * grp, 4 * EG, col, col_ok);
                    continue;
                }
                const float* rcp_col =
                    ((a.epi == 1 || a.epi == 3) && col_ok) ? a.rcp + (int64_t)rbase * a.ld + col % a.ld : nullptr;
                float* c_col = a.C + (int64_t)rbase * a.N + col;
                const int64_t i_col = (int64_t)rbase * a.N + col;     // index of (row rbase, col) in C / u / acc / tmp
#pragma unroll 1
                for (int r0 = 16 * grp; r0 < mr; r0 += 16 * EG) {
                    uint32_t r[16];
                    const uint32_t taddr = tcol + (uint32_t)r0;
                    __syncwarp();                          // reconverge after the lane-dependent stores
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(taddr));
                    // -1/J is loaded while the tensor-memory load is in flight
                    float rc[16];
                    if (rcp_col) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            rc[j] = r0 + j < mr ? __ldg(rcp_col + (int64_t)(r0 + j) * a.ld) : 0.f;
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if constexpr (NT == 2) {
                      if (col_ok && a.epi == 3) {
                        // fused RK stage: k never goes to memory.  Rows go in two halves
                        // of 8 (fewer live registers); the 8 rows of u / acc of a half are
                        // loaded before its first store (the stores may alias them as far
                        // as the compiler knows).
                        const int64_t i0 = i_col + (int64_t)r0 * a.N;
                        const bool need_u = a.rk_mode != 2, need_acc = a.rk_mode != 0;
#pragma unroll
                        for (int h = 0; h < 16; h += 8) {
                            float uu[8], aa[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const bool in = r0 + h + j < mr;
                                uu[j] = (in && need_u) ? __ldg(a.rk_u + i0 + (int64_t)(h + j) * a.N) : 0.f;
                                aa[j] = (in && need_acc) ? a.rk_acc[i0 + (int64_t)(h + j) * a.N] : 0.f;
                            }
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                if (r0 + h + j < mr) {
                                    const float k = -__uint_as_float(r[h + j]) * rc[h + j];
                                    const int64_t i = i0 + (int64_t)(h + j) * a.N;
                                    if (a.rk_mode == 2) {
                                        a.rk_u[i] = aa[j] + a.rk_a * k;
                                    } else {
                                        a.rk_acc[i] = (a.rk_mode == 0 ? uu[j] : aa[j]) + a.rk_a * k;
                                        a.rk_tmp[i] = uu[j] + a.rk_b * k;
                                    }
                                }
                            }
                        }
                        continue;
                      }
                    }
                    if (col_ok) {
                        float* cp = c_col + (int64_t)r0 * a.N;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (r0 + j < mr) {
                                float v = __uint_as_float(r[j]);
                                if (rcp_col) v = -v * rc[j];
                                cp[(int64_t)j * a.N] = v;
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_u32(&bar_tempty[b]));
        }
        if (!ok && tid == 64 + 32 * CONVW) atomicOr(&flags[1], 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ------------------------------------------------------------------ host side
static uint32_t host_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x1000u;                      // round half away from zero at bit 13 (magnitude)
    return u & ~0x1FFFu;
}

static uint16_t host_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static float f_of(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

std::vector<uint8_t> pack_operator(int kind, const std::vector<double>& A, int M, int K1, int K2, int group) {
    const int esz = kind == 0 ? 4 : 2, kce = ROWB / esz;
    const int nch1 = (K1 + kce - 1) / kce, nch2 = (K2 + kce - 1) / kce, nch = nch1 + nch2;
    const int K = K1 + K2;
    std::vector<uint8_t> out;
    // nrb row blocks of rr rows padded to nrp, each: nch chunks of [hi part | lo part]
    const RowBlocks B = row_blocks(M, group);
    for (int rb = 0; rb < B.nrb * B.rr; rb += B.rr) {
        const int nr = std::min(B.rr, M - rb);
        const int nrp = B.nrp, opart = nrp * ROWB;
        const size_t base = out.size();
        out.resize(base + (size_t)nch * 2 * opart, 0);
        for (int c = 0; c < nch; ++c) {
            uint8_t* hi = &out[base + (size_t)c * 2 * opart];
            uint8_t* lo = hi + opart;
            for (int r = 0; r < nrp; ++r)
                for (int kk = 0; kk < kce; ++kk) {
                    const int gr = rb + r;
                    int gk;                                   // operator column of (chunk, kk); -1 = padding
                    if (c < nch1) gk = c * kce + kk < K1 ? c * kce + kk : -1;
                    else gk = (c - nch1) * kce + kk < K2 ? K1 + (c - nch1) * kce + kk : -1;
                    const float v = (r < nr && gk >= 0) ? (float)A[(size_t)gr * K + gk] : 0.f;
                    const int off = core_off(r, kk * esz);
                    if (kind == 0) {
                        uint32_t h = host_tf32(v), l = host_tf32(v - f_of(h));
                        std::memcpy(hi + off, &h, 4);
                        std::memcpy(lo + off, &l, 4);
                    } else {
                        uint16_t h = host_bf16(v);
                        uint16_t l = host_bf16(v - f_of((uint32_t)h << 16));
                        std::memcpy(hi + off, &h, 2);
                        std::memcpy(lo + off, &l, 2);
                    }
                }
        }
    }
    return out;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D map over a row-major FP32 matrix [rows][N], box = kce rows x (nt * 128) columns
static bool make_map(CUtensorMap* m, const float* base, int64_t N, int rows, int kce, int nt) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)N * 4};
    cuuint32_t box[2] = {(cuuint32_t)(BN * nt), (cuuint32_t)kce};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int g_nsm = 0;
static bool g_attr[2] = {false, false};

// Kernel variants (subtiles, converter warps, epilogue groups), by epilogue
// class: the plain / -1/J / RK-stage epilogue (gd = 0) and the gradient
// transform (gd = 2, 3).  Entry 0 of each list is the default rule's choice
// for one subtile, entry 1 for two subtiles.
constexpr int NV0 = 6, NVG = 5;
static const Variant kVar0[NV0] = {{1, 8, 3}, {2, 8, 2}, {1, 8, 2}, {1, 12, 2}, {2, 4, 3}, {1, 4, 3}};
static const Variant kVarG[NVG] = {{1, 4, 4}, {2, 4, 4}, {1, 8, 3}, {1, 8, 4}, {2, 8, 3}};

template <int KIND, int GD, bool M>
static const void* variant_fn_m(int v) {
    if constexpr (GD == 0) {
        switch (v) {
            case 0: return (const void*)tc_gemm_kernel<KIND, 1, 0, 8, 3, M>;
            case 1: return (const void*)tc_gemm_kernel<KIND, 2, 0, 8, 2, M>;
            case 2: return (const void*)tc_gemm_kernel<KIND, 1, 0, 8, 2, M>;
            case 3: return (const void*)tc_gemm_kernel<KIND, 1, 0, 12, 2, M>;
            case 4: return (const void*)tc_gemm_kernel<KIND, 2, 0, 4, 3, M>;
            case 5: return (const void*)tc_gemm_kernel<KIND, 1, 0, 4, 3, M>;
        }
    } else {
        switch (v) {
            case 0: return (const void*)tc_gemm_kernel<KIND, 1, GD, 4, 4, M>;
            case 1: return (const void*)tc_gemm_kernel<KIND, 2, GD, 4, 4, M>;
            case 2: return (const void*)tc_gemm_kernel<KIND, 1, GD, 8, 3, M>;
            case 3: return (const void*)tc_gemm_kernel<KIND, 1, GD, 8, 4, M>;
            case 4: return (const void*)tc_gemm_kernel<KIND, 2, GD, 8, 3, M>;
        }
    }
    return nullptr;
}

template <int KIND, int GD>
static const void* variant_fn(int v, bool multi) {
    return multi ? variant_fn_m<KIND, GD, true>(v) : variant_fn_m<KIND, GD, false>(v);
}

template <int KIND>
static cudaError_t set_smem() {
    for (int multi = 0; multi < 2; ++multi)
        for (int gd : {0, 2, 3})
            for (int v = 0; v < (gd ? NVG : NV0); ++v) {
                const void* f = gd == 0 ? variant_fn<KIND, 0>(v, multi) : gd == 2 ? variant_fn<KIND, 2>(v, multi)
                                                                                  : variant_fn<KIND, 3>(v, multi);
                cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

bool rk_fusable(int M) { return subtiles_for(row_blocks(M, 1).nrp) == 2; }

int variants(int gd, int nrp, int* out) {
    const Variant* tab = gd ? kVarG : kVar0;
    const int n = gd ? NVG : NV0;
    int k = 0;
    for (int v = 0; v < n; ++v)
        if (tab[v].nt == 1 || nrp <= 128) out[k++] = v;
    return k;
}

Variant variant_of(int gd, int v) { return (gd ? kVarG : kVar0)[v]; }

int padded_rows(int M, int group) { return row_blocks(M, group).nrp; }

cudaError_t prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (g_nsm <= 0) g_nsm = 148;
    if ((e = set_smem<0>()) != cudaSuccess || (e = set_smem<1>()) != cudaSuccess) return e;
    g_attr[0] = g_attr[1] = true;
    return encode_fn() ? cudaSuccess : cudaErrorSymbolNotFound;
}

template <int KIND>
static cudaError_t launch(const TcGroup& G, int v, int gd, int nsm, cudaStream_t st) {
    const Variant V = variant_of(gd, v);
    const Layout L = make_layout(KIND, G.nrp, V.nt);
    if (!g_attr[KIND]) {
        cudaError_t e = set_smem<KIND>();
        if (e != cudaSuccess) return e;
        g_attr[KIND] = true;
    }
    const int grid = std::min(G.wstart[G.ng], nsm);
    const int nth = nthreads_for(V.cw, V.eg);
    const bool multi = G.ng > 1;
    const void* f = gd == 0 ? variant_fn<KIND, 0>(v, multi) : gd == 2 ? variant_fn<KIND, 2>(v, multi)
                                                                    : variant_fn<KIND, 3>(v, multi);
    if (!f) return cudaErrorInvalidValue;
    void* args[1] = {(void*)&G};
    return cudaLaunchKernel(f, dim3(grid), dim3(nth), args, (size_t)L.smem, st);
}

// The arguments and tensor maps of one problem of a launch with nt subtiles.
static cudaError_t build_problem(int kind, int epi, const GemmProblem& q, int nt, SubRef sub, int* flags,
                                 long long wait_limit, TcArgs& a, CUtensorMap& m1, CUtensorMap& m2) {
    const int esz = kind == 0 ? 4 : 2, kce = ROWB / esz;
    const GradXform* gx = q.gx;
    const RkFuse* rk = q.rk;
    if (q.N % BN != 0 || q.M <= 0) return cudaErrorInvalidValue;
    if (gx && (gx->ndims < 2 || gx->ndims > 3 || q.M != gx->ndims * gx->nupts || !gx->smat || !q.rcp))
        return cudaErrorInvalidValue;
    const RowBlocks B = row_blocks(q.M, gx ? gx->ndims : 1);
    a.M = q.M;
    a.nrb = B.nrb;
    a.rr = B.rr;
    a.nrp = B.nrp;
    a.nch1 = (q.K1 + kce - 1) / kce;
    a.nch2 = q.K2 > 0 ? (q.K2 + kce - 1) / kce : 0;
    a.subseg = q.subseg;
    a.Apack = (const uint8_t*)q.Apack;
    a.N = q.N;
    a.ld = q.ld;
    a.C = q.C;
    a.epi = epi;
    a.rcp = q.rcp;
    a.sub0 = sub.v[0];
    a.sub1 = sub.v[1];
    a.sub2 = sub.v[2];
    a.sub3 = sub.v[3];
    a.sub4 = sub.v[4];
    a.flags = flags;
    a.limit = wait_limit > 0 ? wait_limit : 4000000000LL;   // SM clock cycles per wait (default ~2 s)
    a.ntiles = (int)((q.N + nt * BN - 1) / (nt * BN));
    a.nwork = a.ntiles * a.nrb;
    a.smat = gx ? gx->smat : nullptr;
    a.gD = gx ? gx->ndims : 0;
    a.gnu = gx ? gx->nupts : 0;
    if (gx) a.epi = 2;
    a.rk_mode = 0;
    a.rk_a = a.rk_b = 0.f;
    a.rk_u = a.rk_acc = a.rk_tmp = nullptr;
    a.rk_nelem = 0;
    if (rk) {
        if (nt != 2) return cudaErrorInvalidValue;          // fused only into the two-subtile kernels
        if (gx || !q.rcp || rk->mode < 0 || rk->mode > 2 || !rk->u || !rk->acc || (rk->mode < 2 && !rk->tmp))
            return cudaErrorInvalidValue;
        a.epi = 3;
        a.rk_mode = rk->mode;
        a.rk_a = rk->a;
        a.rk_b = rk->b;
        a.rk_u = rk->u;
        a.rk_acc = rk->acc;
        a.rk_tmp = rk->tmp;
        a.rk_nelem = rk->nelem;
    }
    // the variables of one element range share the metric terms (adj(J), 1/J)
    // through L2: their column tiles run on neighbouring CTAs at the same time
    const int64_t ld = q.ld, N = q.N;
    a.vinter = (gx && gx->nvars > 1 && ld % (nt * BN) == 0 && N == (int64_t)gx->nvars * ld) ? gx->nvars : 0;
    if (!gx && q.rcp && (epi == 1 || rk) && ld % (nt * BN) == 0 && N % ld == 0 && N / ld > 1) a.vinter = (int)(N / ld);
    if (!make_map(&m1, q.B1, N, q.K1, kce, nt)) return cudaErrorInvalidValue;
    if (q.K2 > 0) {
        if (!make_map(&m2, q.B2, N, q.K2, kce, nt)) return cudaErrorInvalidValue;
    } else {
        m2 = m1;
    }
    return cudaSuccess;
}

cudaError_t gemm_group(int kind, int epi, const GemmProblem* probs, int n, SubRef sub, int* flags, cudaStream_t st,
                       long long wait_limit, int variant) {
    if (!g_nsm) {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
    }
    if (n < 1 || n > MAXG) return cudaErrorInvalidValue;
    // one epilogue class for the whole group
    const int gd = probs[0].gx ? probs[0].gx->ndims : 0;
    int nrp = 0;
    for (int i = 0; i < n; ++i) {
        if ((probs[i].gx ? probs[i].gx->ndims : 0) != gd || (probs[i].rk != nullptr) != (probs[0].rk != nullptr))
            return cudaErrorInvalidValue;
        nrp = std::max(nrp, row_blocks(probs[i].M, gd ? gd : 1).nrp);
    }
    if (variant < 0) variant = subtiles_for(nrp) == 2 ? 1 : 0;          // the default rule
    if (variant >= (gd ? NVG : NV0)) return cudaErrorInvalidValue;
    const Variant V = variant_of(gd, variant);
    if (V.nt == 2 && nrp > 128) return cudaErrorInvalidValue;          // two accumulators per buffer must fit
    TcGroup G;
    std::memset(&G, 0, sizeof(G));
    G.ng = n;
    G.nrp = nrp;
    G.wstart[0] = 0;
    for (int i = 0; i < n; ++i) {
        cudaError_t e = build_problem(kind, epi, probs[i], V.nt, sub, flags, wait_limit, G.p[i], G.m[2 * i],
                                      G.m[2 * i + 1]);
        if (e != cudaSuccess) return e;
        G.wstart[i + 1] = G.wstart[i] + G.p[i].nwork;
    }
    return kind == 0 ? launch<0>(G, variant, gd, g_nsm, st) : launch<1>(G, variant, gd, g_nsm, st);
}

cudaError_t gemm(int kind, int M, int K1, int K2, const void* Apack, const float* B1, const float* B2, int64_t N,
                 float* C, int epi, const float* rcp, int64_t ld, int subseg, SubRef sub, int* flags,
                 cudaStream_t st, const GradXform* gx, const RkFuse* rk, long long wait_limit, int variant) {
    const GemmProblem q{M, K1, K2, Apack, B1, B2, N, C, rcp, ld, subseg, gx, rk};
    return gemm_group(kind, epi, &q, 1, sub, flags, st, wait_limit, variant);
}

int group_max() { return MAXG; }

}  // namespace tc
}  // namespace fr
