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
// Persistent, warp-specialised kernel (one CTA per SM, 10 warps).  The MMA
// M dimension is 128 state columns (one per TMEM lane) and the N dimension is
// the operator's rows (NR, padded to 16; split in two instructions when above
// 256), so each thread of the epilogue owns one state column and every
// operator row of it, and each warp store writes 32 consecutive columns.
//   warp 0      producer: per K chunk, one bulk copy of the packed operator
//               and one 2D TMA load of the FP32 state tile [chunk rows x 128
//               columns]; both complete on the stage's "full" mbarrier;
//   warp 1      MMA issuer (one thread) and owner of tensor memory: three
//               tcgen05.mma per 32-byte K step (state_hi op_hi, state_lo
//               op_hi, state_hi op_lo), committed to the stage's "empty"
//               barrier and, after the last chunk of a column tile, to that
//               tile's accumulator barrier;
//   warps 2-5   converters: read the FP32 tile, subtract the perturbation
//               reference where the rows are solution states, split into
//               hi / lo and write the K-major core-matrix operand layout;
//   warps 6-9   epilogue: tcgen05.ld of the accumulators (one TMEM lane
//               quadrant per warp), optional -1/J scaling, coalesced stores.
// Shared-memory stages form a ring; accumulators are double-buffered in
// tensor memory whenever two fit.  Every mbarrier wait gives up after about
// two seconds of clock cycles and raises the context's timeout flag.
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

constexpr int BN = 128;                        // state columns per tile (MMA M, one per TMEM lane)
constexpr int KSTEPS = 2;                      // 32-byte MMA K steps per chunk
constexpr int ROWB = 32 * KSTEPS;              // bytes of K per operand row per chunk
constexpr int SPART = BN * ROWB;               // one part (hi or lo) of the state operand per chunk
constexpr int NTHREADS = 320;
constexpr int MAX_NST = 6;
constexpr int MAX_NR = 384;                    // operator rows per launch (TMEM: 384 FP32 columns)

// Byte offset of (row r, K byte kb) inside one operand part: core matrices of
// 8 rows x 16 bytes, 2*KSTEPS of them along K, then the next 8-row group.
__host__ __device__ constexpr int core_off(int r, int kb) {
    return ((r >> 3) * (2 * KSTEPS) + (kb >> 4)) * 128 + (r & 7) * 16 + (kb & 15);
}

// operator rows of one launch, padded so that one or two MMA instructions
// (N a multiple of 16, at most 256 each) cover them
__host__ __device__ constexpr int pad_rows(int nr) {
    return nr <= 256 ? (nr + 15) / 16 * 16 : (nr + 31) / 32 * 32;
}

struct Layout {
    int nrp, nsplit, nh;          // padded rows, MMA instructions per K step, N per instruction
    int opart, a_bytes, stg_bytes, off_stg, off_bhi, off_blo, stage, nst, tbuf, smem;
};

__host__ __device__ inline Layout make_layout(int kind, int nr) {
    Layout L;
    L.nrp = pad_rows(nr);
    L.nsplit = L.nrp <= 256 ? 1 : 2;
    L.nh = L.nrp / L.nsplit;
    L.opart = L.nrp * ROWB;
    L.a_bytes = 2 * L.opart;
    const int kce = ROWB / (kind == 0 ? 4 : 2);
    L.stg_bytes = kce * BN * 4;
    L.off_stg = L.a_bytes;
    L.off_bhi = L.off_stg + L.stg_bytes;
    L.off_blo = L.off_bhi + SPART;
    L.stage = L.off_blo + SPART;
    L.nst = (220 * 1024) / L.stage;
    if (L.nst > MAX_NST) L.nst = MAX_NST;
    L.tbuf = 2 * L.nrp <= 512 ? 2 : 1;
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
    int M;              // operator rows handled by this launch
    int row0;           // first operator row of this launch
    int nch1, nch2;     // K chunks of segment 1 (B1) and 2 (B2)
    int subseg;         // segment whose rows get the reference subtracted (0: none)
    const uint8_t* Apack;   // this launch's packed operator: nch chunks of Layout::a_bytes
    int64_t N, ld;
    float* C;
    int epi;
    const float* rcp;
    SubRef sub;
    int* flags;
    long long limit;
    int ntiles;
};

template <int KIND>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_gemm_kernel(const TcArgs a, const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[MAX_NST], bar_conv[MAX_NST], bar_empty[MAX_NST];
    __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2];
    __shared__ uint32_t tmem_holder;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = a.nch1 + a.nch2;
    const Layout L = make_layout(KIND, a.M);
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
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&bar_conv[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[s])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_tfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&bar_tempty[b])));
        }
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
            for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
                const int col0 = tile * BN;
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % L.nst, k = it / L.nst;
                    if (k > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (k - 1) & 1, a.limit)) { ok = false; break; }
                    uint8_t* st = smem + s * L.stage;
                    const uint32_t fb = smem_u32(&bar_full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"((uint32_t)(L.a_bytes + L.stg_bytes))
                                 : "memory");
                    const uint8_t* src = a.Apack + (size_t)c * L.a_bytes;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(st)),
                        "l"(src), "r"((uint32_t)L.a_bytes), "r"(fb)
                        : "memory");
                    const bool seg1 = c < a.nch1;
                    const int row0 = (seg1 ? c : c - a.nch1) * KCE;
                    const CUtensorMap* tm = seg1 ? &tm1 : &tm2;
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
                        "{%2, %3}], [%4];" ::"r"(smem_u32(st + L.off_stg)),
                        "l"(tm), "r"(col0), "r"(row0), "r"(fb)
                        : "memory");
                }
            }
            if (!ok) atomicOr(&a.flags[1], 1);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id = instr_desc<KIND>(L.nh);
            int it = 0, tc = 0;
            for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++tc) {
                const int b = tc % L.tbuf;
                if (!mbar_wait(smem_u32(&bar_tempty[b]), ((tc / L.tbuf) & 1) ^ 1, a.limit)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dbase = tmem + (uint32_t)(b * L.nrp);
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % L.nst, k = it / L.nst;
                    if (!mbar_wait(smem_u32(&bar_conv[s]), k & 1, a.limit)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = smem_u32(smem + s * L.stage);
                    const uint32_t o_hi = st, o_lo = st + L.opart;            // operator parts (MMA B)
                    const uint32_t s_hi = st + L.off_bhi, s_lo = st + L.off_blo;  // state parts (MMA A)
#pragma unroll
                    for (int j = 0; j < KSTEPS; ++j) {
                        const uint32_t o = 2 * j * 128;
                        const uint32_t first = (c == 0 && j == 0) ? 0u : 1u;
                        for (int h = 0; h < L.nsplit; ++h) {
                            const uint32_t d = dbase + (uint32_t)(h * L.nh);
                            const uint32_t ro = (uint32_t)(h * L.nh / 8) * (2 * KSTEPS * 128);   // row-group offset
                            mma<KIND>(d, make_desc(s_hi + o), make_desc(o_hi + ro + o), id, first);
                            mma<KIND>(d, make_desc(s_lo + o), make_desc(o_hi + ro + o), id, 1u);
                            mma<KIND>(d, make_desc(s_hi + o), make_desc(o_lo + ro + o), id, 1u);
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
            if (!ok) atomicOr(&a.flags[1], 1);
        }
    } else if (warp < 6) {
        // ---------------------------------------------------------- converters
        const int ct = tid - 64;                       // state column within the tile = MMA A row
        int it = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
            const int64_t gc = (int64_t)tile * BN + ct;
            const float subv = gc < a.N ? a.sub.v[gc / a.ld] : 0.f;
            for (int c = 0; c < nch; ++c, ++it) {
                const int s = it % L.nst, k = it / L.nst;
                if (!mbar_wait(smem_u32(&bar_full[s]), k & 1, a.limit)) { ok = false; break; }
                uint8_t* st = smem + s * L.stage;
                const float* stg = (const float*)(st + L.off_stg);
                const bool seg1 = c < a.nch1;
                const float sv = (a.subseg == (seg1 ? 1 : 2)) ? subv : 0.f;
#pragma unroll
                for (int g = 0; g < ROWB / 16; ++g) {
                    constexpr int PER = 16 / ESZ;
                    float x[PER];
#pragma unroll
                    for (int q = 0; q < PER; ++q) x[q] = stg[(g * PER + q) * BN + ct] - sv;
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
                    *(uint4*)(st + L.off_bhi + core_off(ct, 16 * g)) = h;
                    *(uint4*)(st + L.off_blo + core_off(ct, 16 * g)) = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&bar_conv[s]));
            }
        }
        if (!ok && ct == 0) atomicOr(&a.flags[1], 1);
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                        // TMEM lane quadrant of this warp
        int tc = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++tc) {
            const int b = tc % L.tbuf;
            if (!mbar_wait(smem_u32(&bar_tfull[b]), (tc / L.tbuf) & 1, a.limit)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int64_t col = (int64_t)tile * BN + q * 32 + lane;    // this thread's state column
            const float* rcp_col = a.epi == 1 ? a.rcp + (int64_t)a.row0 * a.ld + col % a.ld : nullptr;
            float* c_col = a.C + (int64_t)a.row0 * a.N + col;
            // -1/J of the next 16 rows is loaded before the previous 16 are stored, so the
            // loads never wait behind stores they might alias
            float rc[16];
            if (a.epi == 1) {
#pragma unroll
                for (int j = 0; j < 16; ++j) rc[j] = j < a.M ? __ldg(rcp_col + (int64_t)j * a.ld) : 0.f;
            }
#pragma unroll 1
            for (int r0 = 0; r0 < a.M; r0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * L.nrp + r0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                float rn[16];
                if (a.epi == 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        rn[j] = r0 + 16 + j < a.M ? __ldg(rcp_col + (int64_t)(r0 + 16 + j) * a.ld) : 0.f;
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float* cp = c_col + (int64_t)r0 * a.N;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (r0 + j < a.M) {
                        float v = __uint_as_float(r[j]);
                        if (a.epi == 1) v = -v * rc[j];
                        cp[(int64_t)j * a.N] = v;
                    }
                }
                if (a.epi == 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) rc[j] = rn[j];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_u32(&bar_tempty[b]));
        }
        if (!ok && tid == 192) atomicOr(&a.flags[1], 1);
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

std::vector<uint8_t> pack_operator(int kind, const std::vector<double>& A, int M, int K1, int K2) {
    const int esz = kind == 0 ? 4 : 2, kce = ROWB / esz;
    const int nch1 = (K1 + kce - 1) / kce, nch2 = (K2 + kce - 1) / kce, nch = nch1 + nch2;
    const int K = K1 + K2;
    std::vector<uint8_t> out;
    // row blocks of at most MAX_NR rows, each: nch chunks of [hi part | lo part]
    for (int rb = 0; rb < M; rb += MAX_NR) {
        const int nr = std::min(MAX_NR, M - rb);
        const int nrp = pad_rows(nr), opart = nrp * ROWB;
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

// 2D map over a row-major FP32 matrix [rows][N], box = kce rows x 128 columns
static bool make_map(CUtensorMap* m, const float* base, int64_t N, int rows, int kce) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)N * 4};
    cuuint32_t box[2] = {(cuuint32_t)BN, (cuuint32_t)kce};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int g_nsm = 0;
static bool g_attr[2] = {false, false};

cudaError_t prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (g_nsm <= 0) g_nsm = 148;
    if ((e = cudaFuncSetAttribute(tc_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024)) !=
        cudaSuccess)
        return e;
    g_attr[0] = g_attr[1] = true;
    return encode_fn() ? cudaSuccess : cudaErrorSymbolNotFound;
}

template <int KIND>
static cudaError_t launch(const TcArgs& a, const CUtensorMap& m1, const CUtensorMap& m2, int nsm, cudaStream_t st) {
    const Layout L = make_layout(KIND, a.M);
    if (!g_attr[KIND]) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             225 * 1024);
        if (e != cudaSuccess) return e;
        g_attr[KIND] = true;
    }
    const int grid = std::min(a.ntiles, nsm);
    tc_gemm_kernel<KIND><<<grid, NTHREADS, L.smem, st>>>(a, m1, m2);
    return cudaGetLastError();
}

cudaError_t gemm(int kind, int M, int K1, int K2, const void* Apack, const float* B1, const float* B2, int64_t N,
                 float* C, int epi, const float* rcp, int64_t ld, int subseg, SubRef sub, int* flags,
                 cudaStream_t st) {
    if (!g_nsm) {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
    }
    const int nsm = g_nsm;
    if (N % BN != 0) return cudaErrorInvalidValue;
    const int esz = kind == 0 ? 4 : 2, kce = ROWB / esz;
    CUtensorMap m1, m2;
    if (!make_map(&m1, B1, N, K1, kce)) return cudaErrorInvalidValue;
    if (K2 > 0) {
        if (!make_map(&m2, B2, N, K2, kce)) return cudaErrorInvalidValue;
    } else {
        m2 = m1;
    }
    TcArgs a;
    a.nch1 = (K1 + kce - 1) / kce;
    a.nch2 = K2 > 0 ? (K2 + kce - 1) / kce : 0;
    a.subseg = subseg;
    a.N = N;
    a.ld = ld;
    a.C = C;
    a.epi = epi;
    a.rcp = rcp;
    a.sub = sub;
    a.flags = flags;
    a.limit = 4000000000LL;                  // ~2 s of SM clock cycles per wait
    a.ntiles = (int)(N / BN);
    size_t off = 0;
    for (int rb = 0; rb < M; rb += MAX_NR) {
        a.M = std::min(MAX_NR, M - rb);
        a.row0 = rb;
        a.Apack = (const uint8_t*)Apack + off;
        cudaError_t e = kind == 0 ? launch<0>(a, m1, m2, nsm, st) : launch<1>(a, m1, m2, nsm, st);
        if (e != cudaSuccess) return e;
        off += (size_t)(a.nch1 + a.nch2) * 2 * pad_rows(a.M) * ROWB;
    }
    return cudaSuccess;
}

}  // namespace tc
}  // namespace fr
