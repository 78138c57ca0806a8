// noalloc.cu -- svd_truncate_noalloc: the SVD + entropy + truncation of
// svd_truncate for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running where the device memory
// is owned by another component (a framework's caching pool that must see
// every allocation, or a fixed memory budget sized ahead of time), and
// time-critical loops where an allocation, which can synchronise the whole
// device, is not acceptable.  This entry point performs no allocation of any
// kind: its scratch (the Jacobi vectors, rotations, norms, permutation,
// barrier words and the small result record) lives in a file-scope device
// array of fixed size, which every GPU that loads the library holds until the
// process exits.
#include "common.cuh"
#include "ctrl.cuh"

#include <mutex>

namespace dmrg {
namespace {

// Largest supported problem: m, n <= kNoAllocMaxDim.
constexpr int kNoAllocMaxDim = 256;
// 2 * 8 * 256 * 256 bytes (vectors and rotations) plus norms, permutation,
// barrier words and the result record, each rounded to 256 bytes.
constexpr size_t kNoAllocScratchBytes = 1114112;   // 1088 KiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on `device`, looked up once per
// device with that device current (host code cannot use the symbol itself).
dmrg_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return DMRG_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        int prev = 0;
        DMRG_CUDA(cudaGetDevice(&prev));
        if (prev != device) DMRG_CUDA(cudaSetDevice(device));
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess || !p) {
            std::fprintf(stderr, "dmrg: cudaGetSymbolAddress of the no-alloc scratch failed: %s\n",
                         cudaGetErrorString(e));
            return DMRG_ECUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return DMRG_OK;
}

}  // namespace
}  // namespace dmrg

using namespace dmrg;

extern "C" dmrg_status svd_truncate_noalloc(dmrg_ctx *ctx, const double *theta_dev, int m, int n, int chi_max,
                                            double eps, double *U_dev, double *s_dev, double *Vt_dev, int *k_out,
                                            double *S_out, double *trunc_err_out)
{
    if (!ctx || !theta_dev || !U_dev || !s_dev || !Vt_dev || m < 1 || n < 1 || chi_max < 1 || !(eps >= 0.0))
        return DMRG_EINVAL;
    if (m > kNoAllocMaxDim || n > kNoAllocMaxDim) {
        std::fprintf(stderr, "dmrg: svd_truncate_noalloc supports m, n <= %d (got %d x %d); use svd_truncate\n",
                     kNoAllocMaxDim, m, n);
        return DMRG_EINVAL;
    }
    const int r = m < n ? m : n, l = m < n ? n : m;
    const size_t work = al256(svd_work_bytes_base(r, l));
    const size_t need = work + al256(sizeof(BondResult)) + al256(sizeof(int) * 4);
    if (need > kNoAllocScratchBytes) {
        std::fprintf(stderr, "dmrg: svd_truncate_noalloc scratch too small (%zu > %zu bytes)\n", need,
                     kNoAllocScratchBytes);
        return DMRG_EINVAL;
    }
    void *base = nullptr;
    DMRG_TRY(scratch_address(ctx->device, &base));
    char *b = static_cast<char *>(base);
    BondResult *res = reinterpret_cast<BondResult *>(b + work);
    int *info = reinterpret_cast<int *>(b + work + al256(sizeof(BondResult)));
    // The Jacobi load kernel clears the barrier words and rotation counters it
    // reuses from the previous call; everything else is written before it is read.
    DMRG_TRY(svd_jacobi(ctx, theta_dev, m, n, U_dev, s_dev, Vt_dev, b, ctx->jacobi_max_sweeps, info, 0));
    dmrg_params p{};
    p.eps_trunc = eps;
    p.chi_min = 1;
    p.chi_max = chi_max;
    p.multiplet_guard = 0;
    p.ctrl = DMRG_CTRL_FIXED;
    DMRG_TRY(launch_decide(ctx, s_dev, r, nullptr, p, 0, chi_max, nullptr, 0, 1, 0, nullptr, res, nullptr, 0,
                           (double)r * 2.220446049250313e-16));
    DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_d, res, sizeof(BondResult), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_i + 40, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    BondResult br;
    std::memcpy(&br, ctx->h_pinned_d, sizeof(BondResult));
    if (k_out) *k_out = br.k;
    if (S_out) *S_out = br.S;
    if (trunc_err_out) *trunc_err_out = br.eps;
    dmrg_status ds = dmrg_get_status(ctx);
    if (ctx->h_pinned_i[40] < 0) return DMRG_ENOCONV;
    return ds == DMRG_ENOCONV ? DMRG_OK : ds;
}
