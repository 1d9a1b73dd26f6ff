// vie_apply_noalloc: the FP32 operator application of vie_apply_device with
// its FFT workspace taken from a fixed, file-scope device array instead of
// memory allocated by the library.
//
// Who needs it: callers whose device memory is owned by someone else -- a
// framework's caching allocator, a memory pool sized at start-up, an
// embedded or real-time host loop -- and that therefore must not have the
// library call cudaMalloc/cudaFree (or any allocating routine) behind their
// back.  With this entry point the caller owns every input and output buffer,
// the handle owns what vie_setup allocated once, and the per-call scratch is
// the static array below.
//
// Costs and limits: the array (NOALLOC_SCRATCH_BYTES, 64 MiB) exists on every
// GPU that loads the library, for as long as the process runs.  One RHS of the
// operator needs 3*n0*n1*P2 + 3*n0*P1*P2 complex64 words of workspace (P the
// padded sizes); grids whose single-RHS workspace exceeds the array are
// rejected with VIE_EINVAL (64^3 grids fit, 128^3 grids do not).  Only the
// power-of-two padded sizes of the register FFT path are supported.
#include <cstring>
#include <mutex>

#include "vie_internal.cuh"

namespace vie {
Operator* handle_operator(vie_handle* hd);
int handle_device(const vie_handle* hd);
}

using namespace vie;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 64ull << 20;
constexpr int NOALLOC_MAX_RHS = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Every call shares this array; it keeps the previous call's contents.  No
// part of it needs to start at zero: each pass fully overwrites the region it
// later reads (zero padding is produced inside the FFT kernels).
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
// RHS index list 0, 1, ..., NOALLOC_MAX_RHS-1 used by the batched launches
__device__ __align__(256) int g_noalloc_iota[NOALLOC_MAX_RHS];

struct DeviceScratch {
    bool ready = false;
    unsigned char* scratch = nullptr;
    int* iota = nullptr;
};
DeviceScratch g_dev[NOALLOC_MAX_DEVICES];
std::mutex g_mu;

// Per device, with that device current: look up the device addresses of the
// two arrays (in host code their names only stand for them) and fill the
// index list.  Runs on the first call on each device.
int noalloc_setup(int dev, DeviceScratch** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(VIE_EINVAL, "device ordinal out of range");
    DeviceScratch& d = g_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_noalloc_iota);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(index list)");
        int host[NOALLOC_MAX_RHS];
        for (int i = 0; i < NOALLOC_MAX_RHS; ++i) host[i] = i;
        e = cudaMemcpyToSymbol(g_noalloc_iota, host, sizeof(host));
        if (e != cudaSuccess) return cuda_fail(e, "index list upload");
        d.scratch = static_cast<unsigned char*>(p);
        d.iota = static_cast<int*>(q);
        d.ready = true;
    }
    *out = &d;
    return VIE_OK;
}

}  // namespace

extern "C" int vie_apply_noalloc(vie_handle* hd, const void* w_dev, void* y_dev, int n_rhs) {
    if (!hd || !w_dev || !y_dev) return fail(VIE_EINVAL, "NULL argument");
    if (n_rhs < 1 || n_rhs > NOALLOC_MAX_RHS)
        return fail(VIE_EINVAL, "n_rhs must be in 1.." + std::to_string(NOALLOC_MAX_RHS));
    Operator& op = *handle_operator(hd);
    if (op.disc) return fail(VIE_EINVAL, "vie_apply_noalloc covers the D1 discretisation only");
    // one voxel map and one contrast for every slot (a plain vie_setup handle)
    if (op.idx_stride != 0 || op.chi_cs != 0)
        return fail(VIE_EINVAL, "vie_apply_noalloc needs one shared voxel map and contrast per handle");
    if (op.fft_path != 0)
        return fail(VIE_EINVAL, "vie_apply_noalloc runs the register FFT passes only; the handle is set to the "
                                "generic path (vie_set_fft_path)");
    const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2];
    const int P0 = op.P[0], P1 = op.P[1], P2 = op.P[2];
    if (!fast_length(P0) || !fast_length(P1) || !fast_length(P2))
        return fail(VIE_EINVAL, "vie_apply_noalloc needs power-of-two padded sizes (16..512) on every axis");
    const size_t slotA = sizeof(c32) * 3ull * n0 * n1 * P2;
    const size_t slotA_al = (slotA + 255) & ~(size_t)255;
    const size_t slotB = sizeof(c32) * 3ull * n0 * P1 * P2;
    const size_t per = slotA_al + slotB;
    if (per > NOALLOC_SCRATCH_BYTES)
        return fail(VIE_EINVAL, "grid too large for the fixed scratch: one RHS needs " + std::to_string(per) +
                                    " bytes, the array holds " + std::to_string(NOALLOC_SCRATCH_BYTES));
    // the handle's device, as every other entry point: its stream, maps and
    // spectra live there, so the scratch address must be that device's too
    const int dev = handle_device(hd);
    VIE_CUDA(cudaSetDevice(dev));
    DeviceScratch* ds = nullptr;
    VIE_TRY(noalloc_setup(dev, &ds));
    const int cap = (int)(NOALLOC_SCRATCH_BYTES / (slotA_al + slotB));
    const long long n3 = 3 * op.Nb;
    const c32* w = static_cast<const c32*>(w_dev);
    c32* y = static_cast<c32*>(y_dev);
    cudaStream_t s = op.stream;
    for (int s0 = 0; s0 < n_rhs; s0 += cap) {
        const int ns = std::min(cap, n_rhs - s0);
        c32* A = reinterpret_cast<c32*>(ds->scratch);
        c32* B = reinterpret_cast<c32*>(ds->scratch + ((ns * slotA + 255) & ~(size_t)255));
        const int* list = ds->iota + s0;
        const long long nlines = (long long)ns * 3 * n0 * n1;
        VIE_TRY(fast_zfwd(w, n3, list, op.idx_map, A, n0, n1, n2, op.Nb, nlines, P2, op.ax[2].roots32, s,
                          op.idx_stride));
        VIE_TRY(fast_axis(A, B, (long long)ns * 3 * n0, n1, P1, P2, P1, op.ax[1].roots32, false, s));
        VIE_TRY(fast_xfused(B, n0, (long long)P1 * P2, P0, P1, P2, op.khat32, op.H, op.ax[0].roots32, ns, s));
        VIE_TRY(fast_axis(B, A, (long long)ns * 3 * n0, P1, n1, P2, P1, op.ax[1].roots32, true, s));
        VIE_TRY(fast_zinv(A, w, n3, y, n3, list, op.idx_map, op.chi32, n0, n1, n2, op.Nb, nlines, P2,
                          op.ax[2].roots32, s, op.chi_cs, op.idx_stride));
        count_launch(5);
        VIE_CUDA(cudaGetLastError());
    }
    return VIE_OK;
}
