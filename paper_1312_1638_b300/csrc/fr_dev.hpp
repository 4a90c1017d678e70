// Device-side state of an FR context and the kernel launchers (CUDA).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace fr {

// Physical / numerical parameters as passed to kernels (Sec. 4, App. C).
struct DevParams {
    double gamma, mu, prandtl, beta, tau;
    double bc_rho, bc_v[3], bc_p, outflow_p, wall_cpTw, wall_v[3], wall2_v[3];
    // perturbation form: reference state at rest (all zero = plain form)
    double ref_rho, ref_E, ref_p, ref_h;
};

// One element block on the device.  Buffers hold T = double (FP64) or float.
struct DevBlock {
    int etype = 0, nupts = 0, nfpts = 0, nvars = 0;
    int64_t nelem = 0, ld = 0;
    void* smat = nullptr;      // adj(J): [ndims*ndims][nupts][ld]
    void* rcpdjac = nullptr;   // 1/det J: [nupts][ld]
    double* wdet = nullptr;    // FP64 quadrature weight * det J: [nupts][ld]
    void* Uf = nullptr;        // [nfpts][nvars][ld]   U^(f), then D~ in place
    void* Q = nullptr;         // [ndims*nupts][nvars][ld]  Q~ -> Q -> F~ in place
    void* Qf = nullptr;        // [ndims*nfpts][nvars][ld]  C^(f), then Q^(f)  (NS)
    void* opM0 = nullptr;      // M0: nfpts x nupts
    void* opQ = nullptr;       // [M6 | M4 - M6 M0]: ndims*nupts x (nfpts + nupts)
    void* opR = nullptr;       // [M3 | M1 - M3 M2]: nupts x (nfpts + ndims*nupts)
    void* tcM0 = nullptr;      // the same three operators packed for the tensor-core GEMM
    void* tcQ = nullptr;       // (split-precision modes only)
    void* tcR = nullptr;
    // adjoint: transposed operators and scratch
    void* opM3T = nullptr;     // M3^T: nfpts x nupts
    void* opM132T = nullptr;   // (M1 - M3 M2)^T: ndims*nupts x nupts
    void* opM0T = nullptr;     // M0^T: nupts x nfpts
    void* opM6T = nullptr;     // (NS) M6^T: nfpts x ndims*nupts
    void* opOutT = nullptr;    // (NS) [M0^T | (M4 - M6 M0)^T]: nupts x (nfpts + ndims*nupts)
    void* tcM3T = nullptr;
    void* tcM132T = nullptr;
    void* tcM0T = nullptr;
    void* tcM6T = nullptr;
    void* tcOutT = nullptr;
    void* adj_mu = nullptr;    // [nupts][nvars][ld]
    void* adj_uf = nullptr;    // [nfpts][nvars][ld]
    void* adj_g = nullptr;     // (NS) [ndims*nupts][nvars][ld]: g_F
    void* adj_x = nullptr;     // (NS) [ndims*nupts][nvars][ld]: M0^T applied to the flux-point gradient adjoint
    void* stage = nullptr;     // device staging for fr_rhs_host: [nupts][nvars][ld]
    void* rk_acc = nullptr;    // RK4 registers
    void* rk_tmp = nullptr;
    void* dp_k = nullptr;          // DOPRI5: 7 slope arrays, one state size apart
    void* dp_y = nullptr;          // DOPRI5: stage input / new solution
    // tensor-core kernel variant of each operator product (TUNE_*; -1: the default rule)
    int tune[4] = {-1, -1, -1, -1};
    // M0 in structured form (every row with at most sp_nnz <= 8 nonzeros; 0: dense):
    // column indices [nfpts][sp_nnz] and values (T) of each row, zero-padded
    int sp_nnz = 0;
    int* sp_idx = nullptr;
    void* sp_val = nullptr;
    // the corrected-gradient operator [M6 | M4 - M6 M0] in structured form
    // (NS; rows (i, s), [ndims*nupts][gs_nnz] SpPair<T> entries over the columns
    // [nfpts + nupts], zero-padded; 0: dense)
    int gs_nnz = 0;
    void* gs_ent = nullptr;
    // the divergence operator [M3 | M1 - M3 M2] in the same form (rows s,
    // [nupts][ds_nnz] over the columns [nfpts + ndims*nupts]; at most 24)
    int ds_nnz = 0;
    void* ds_ent = nullptr;
    // tensor-line form (quadrilaterals, hexahedra): n = p+1 points per line (0:
    // none), whether the gradient / divergence operators take it, their n x (n+2)
    // line matrices, and the two flux points ending each line, [ndims n^(ndims-1)][2]
    int ln_n = 0;
    bool ln_grad = false, ln_div = false;
    double ln_A[48] = {}, ln_B[48] = {};
    int* ln_fl = nullptr;
    // M0 in line form: the rows of a line's two end flux points, each over the
    // line's n points ([2][n]: the xi_i = -1 end, then +1); the gradient kernel
    // then also forms Q^(f)
    bool ln_interp = false;
    double ln_I0[12] = {};
    // the adjoint's operators (adjoint_gemm `which` 1..4: M3^T, (M1 - M3 M2)^T,
    // M0^T, M6^T) in structured form: [rows][nnz] columns and values (at most
    // 8 nonzeros per row); which 5, [M0^T | (M4 - M6 M0)^T]: packed SpPair<T>
    // entries (at most 24); nnz 0: dense
    int adj_nnz[6] = {};
    int* adj_idx[6] = {};
    void* adj_val[6] = {};
    void* adj_ent = nullptr;
};

// one nonzero of a structured operator row: value and column, packed so that
// one 8-byte (FP32) or 16-byte (FP64) load fetches both
template <typename T>
struct alignas(sizeof(T) == 8 ? 16 : 8) SpPair {
    T v;
    int k;
};

// operator products whose kernel variant can be chosen (DevBlock::tune)
enum TuneSlot { TUNE_DISU = 0, TUNE_TGRADU, TUNE_GRADFPTS, TUNE_TDIVF, TUNE_N };

struct DevPairGroup {          // interior pairs between block bL and block bR
    int bL = 0, bR = 0;
    int64_t n = 0;
    uint32_t* offL = nullptr;  // fpt*nvars*ld + elem in the L block's flux-point arrays
    uint32_t* offR = nullptr;
    void* nrm = nullptr;       // [ndims][n] unit normal of L (T)
    void* magL = nullptr;      // [n] J^(f) n^(f) of L (T)
    void* magR = nullptr;
};

// Cross-partition pairs (Sec. 3.6 "mpi" interfaces) with one neighbour rank,
// one of my blocks and one orientation: my side is the global L side
// (mine_L) or the R side; the other side's values arrive in the neighbour's
// exchange buffers at the pairs' slots.
struct DevMpiGroup {
    int nb = 0;                // index into DevCtx::nbrs
    int b = 0;                 // my block
    bool mine_L = true;
    int64_t n = 0;
    uint32_t* off = nullptr;   // my flux-point offsets fpt*nvars*ld + elem
    uint32_t* slot = nullptr;  // slot of each pair in the exchange buffers
    void* nrm = nullptr;       // [ndims][n] unit normal of the global L side (T)
    void* magL = nullptr;
    void* magR = nullptr;
};

// exchange buffers with one neighbour rank: U^(f) [nvars][nslots], Q^(f) [ndims][nvars][nslots]
struct DevNeighbour {
    int q = 0;
    int64_t nslots = 0;
    void* send_u = nullptr;
    void* recv_u = nullptr;
    void* send_q = nullptr;
    void* recv_q = nullptr;
};

struct DevBndGroup {           // boundary flux points of one block and one type
    int b = 0, bctype = 0;
    int64_t n = 0;
    uint32_t* off = nullptr;
    void* nrm = nullptr;
    void* mag = nullptr;
};

// Kernel-level timing: CUDA events recorded on the launch stream around each
// kernel when profiling is enabled.
enum KernelId {
    K_DISU = 0, K_COMM_SOL, K_COMM_SOL_BC, K_TGRADU, K_GRADCORU, K_GRADFPTS, K_TDISF, K_COMM_FLUX,
    K_COMM_FLUX_BC, K_TDIVF, K_RK_STAGE, K_NKERNELS
};
extern const char* const kKernelNames[K_NKERNELS];

struct ProfRec {
    int id;
    cudaEvent_t a, b;
};

struct DevCtx {
    bool prof = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    int device = -1;
    int ndims = 0, nvars = 0, system = 0, precision = 0, order = 0;
    DevParams prm{};
    std::vector<DevBlock> blocks;
    std::vector<DevPairGroup> pgroups;
    std::vector<DevBndGroup> bgroups;
    std::vector<DevNeighbour> nbrs;   // partitioned context: neighbour ranks
    std::vector<DevMpiGroup> mgroups;
    int* flags = nullptr;          // [0] non-finite seen, [1] timeout
    long long tc_wait_limit = 0;   // tensor-core GEMM wait limit in SM cycles (0: about two seconds)
    bool group_blocks = true;      // tensor-core products of all element blocks in one launch per stage
    bool structured_interp = true; // M0 products through the structured kernel where M0 allows
    // corrected gradient / divergence through a structured kernel where the
    // operator allows: 0 never (dense products), 1 the tensor-line kernel, else
    // the row-wise one, 2 the row-wise kernel
    int structured_grad = 1;
    int structured_div = 1;
    bool structured_adjoint = true; // the adjoint's operator products through the structured kernels where they allow
    double* partial = nullptr;     // reduction scratch
    int64_t npartial = 0;
};

// profiling helpers (no-ops when c.prof is false)
void prof_begin(DevCtx& c, int id, cudaStream_t st);
void prof_end(DevCtx& c, cudaStream_t st);
// drain: per kernel id, launches and total ms since the last drain (synchronises)
cudaError_t prof_drain(DevCtx& c, int64_t* launches, double* ms);
void prof_free(DevCtx& c);

// RHS r = R(u) for every block (precision and dimension dispatched inside).
cudaError_t launch_rhs(DevCtx& c, void* const* u, void* const* r, cudaStream_t st);
// out = (dR/du)^T lam; scratch must be allocated (adj_mu, adj_uf; NS also adj_g, adj_x)
cudaError_t launch_adjoint_rhs(DevCtx& c, void* const* u, void* const* lam, void* const* out, cudaStream_t st);
// operator product used by the adjoint: which = 0: M0 u (plain), 1: M3^T x, 2: (M1-M3M2)^T x, 3: M0^T x,
// (NS) 4: M6^T x, 5: M0^T x + (M4 - M6 M0)^T y with y = B2
cudaError_t adjoint_gemm(DevCtx& c, int which, int b, const void* B, void* C, cudaStream_t st,
                         const void* B2 = nullptr);
// RK4 adjoint: lam (dK/du_N on entry) becomes dK/du_0; ck: ceil(nsteps/every)
// state slots, blk: `every` slots, tmp: 8 slots (each [block] -> device buffer)
cudaError_t launch_rk4_adjoint(DevCtx& c, void* const* u0, void* const* lam, double dt, int nsteps, int every,
                               const std::vector<std::vector<void*>>& ck, const std::vector<std::vector<void*>>& blk,
                               const std::vector<std::vector<void*>>& tmp, cudaStream_t st);
// classical RK4, nsteps steps of dt, in place on u
cudaError_t launch_rk4(DevCtx& c, void* const* u, double dt, int nsteps, cudaStream_t st);
// whether block b's divergence product carries the RK stage (tensor-core paths)
bool tdivf_fused(const DevCtx& c, const DevBlock& B);
// candidate kernel variants of operator product `slot` of block B (at most 8), count returned
int tune_candidates(const DevCtx& c, const DevBlock& B, int slot, int* out);
// RHS phases of a partitioned context (all of them for an ordinary one):
// A = disu + pack U^(f); B1 = common solution, interior and boundary pairs;
// B2 = common solution at partition pairs, gradients, pack Q^(f);
// C1 = transformed flux, common flux at interior and boundary pairs;
// C2 = common flux at partition pairs, divergence (+ energy-split correction)
enum RhsPhase { PH_A = 1, PH_B1 = 2, PH_B2 = 4, PH_C1 = 8, PH_C2 = 16, PH_ALL = 31 };
cudaError_t launch_rhs_phases(DevCtx& c, void* const* u, void* const* r, int phases, cudaStream_t st);
cudaError_t launch_euler(DevCtx& c, void* const* u, double dt, int nsteps, cudaStream_t st);
cudaError_t launch_dopri5(DevCtx& c, void* const* u, double dt, int nsteps, double atol, double rtol, double* err,
                          cudaStream_t st);
// FP64 weighted totals per variable
cudaError_t launch_sum_weighted(DevCtx& c, void* const* u, double* host_out, cudaStream_t st);
cudaError_t launch_check_finite(DevCtx& c, void* const* u, cudaStream_t st);
// FP32 and FP64 FMA throughput of the current device (TFLOP/s), synchronous
cudaError_t measure_fma(double* fp32_tflops, double* fp64_tflops);
// raise the structured interpolation kernel's shared-memory limit for an
// element type (nupts solution, nfpts flux points, nnz nonzeros per row)
cudaError_t interp_prepare(int nupts, int nfpts, int nnz, bool fp64);
// the same for the structured corrected-gradient kernel
cudaError_t grad_prepare(int nupts, int nfpts, int ndims, int nnz, bool fp64);
cudaError_t div_prepare(int nupts, int nfpts, int ndims, int nnz, bool fp64);
// whether the structured product kernels take an M x K operator with nnz
// nonzeros per row (kind 0: at most 8; kind 1: at most 24 over two stacked
// sources), raising their shared-memory limits if so
bool sparse_prepare(int kind, int M, int K, int nnz, bool fp64);
// the tensor-line kernels: kind 0 gradient, 1 divergence; n = p+1
cudaError_t line_prepare(int kind, int ndims, int n, int nfpts, bool fp64);
// look up the allocation-free RK4's fixed device array on `device` (current),
// reserving it there; failures are left for fr_rk4_noalloc to report
void noalloc_prepare(int device);

}  // namespace fr

// Internal accessors of the opaque context for entry points defined outside
// fr_api.cu (implemented there).
struct fr_ctx;
namespace fr {
DevCtx* ctx_dev(fr_ctx* c);
void ctx_set_error(fr_ctx* c, const char* msg);
bool ctx_is_part(const fr_ctx* c);   // built by fr_setup_part
}  // namespace fr
