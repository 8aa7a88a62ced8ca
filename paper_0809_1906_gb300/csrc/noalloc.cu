// noalloc.cu -- bc_run_noalloc: betweenness with no allocation at all.
//
// Some callers cannot allocate device memory: code that runs while a custom
// allocator or memory pool owns the whole device, plug-ins whose host process
// forbids cudaMalloc after start-up, or setups that must keep a fixed memory
// footprint. For them this entry point runs the same batched multi-source
// kernels as bc_run (msbfs.cu) with every scratch buffer carved out of one
// fixed array in device global memory, declared below. The caller passes the
// graph, the source list and the output (all device pointers); nothing else
// is allocated: no cudaMalloc, cudaFree, pinned host memory, events or host
// heap.
//
// The array is a file-scope __device__ variable, so every GPU on which the
// library is loaded holds BC_NOALLOC_SCRATCH_BYTES of it until the process
// exits. In host code its name is only a host-side stand-in; the device
// address is obtained with cudaGetSymbolAddress once per device (on the first
// call made with that device current) and cached.
#include <cuda_runtime.h>

#include <mutex>

#include "bc_internal.cuh"

namespace {

// The limits below fix the array size: with B = 32 sources per batch, a
// batch needs per vertex 256 B of path counts, 128 B of masked count rows
// (two levels), 256 B of masked dependency rows (two levels), 4 B of
// frontier bits per level (64 levels), 8 B of visited bits and 16 B of work
// item; plus the bitmaps and the control blocks.
constexpr int kW = 1;   // 32 sources per batch
constexpr int kB = 32 * kW;
constexpr int kMaxN = BC_NOALLOC_MAX_N;
constexpr int kLcap = BC_NOALLOC_MAX_LEVELS + 2;  // levels 0..depth, plus the empty next frontier
constexpr int kNw32 = (kMaxN + 31) / 32;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffSigma = 0;
constexpr size_t kOffS = align256(kOffSigma + (size_t)kMaxN * kB * sizeof(uint64_t));
constexpr size_t kOffWide = align256(kOffS + (size_t)2 * kMaxN * kB * sizeof(uint16_t));
constexpr size_t kOffCval = align256(kOffWide + (size_t)kLcap * sizeof(uint32_t));
constexpr size_t kOffF = align256(kOffCval + (size_t)2 * kMaxN * kB * sizeof(float));
constexpr size_t kOffUfr = align256(kOffF + (size_t)kLcap * kMaxN * kW * sizeof(uint32_t));
constexpr size_t kOffV = align256(kOffUfr + (size_t)kLcap * kNw32 * sizeof(uint32_t));
constexpr size_t kOffItems = align256(kOffV + (size_t)2 * kMaxN * kW * sizeof(uint32_t));
constexpr size_t kOffSrc = align256(kOffItems + (size_t)4 * kMaxN * sizeof(int32_t));
constexpr size_t kOffCtl = align256(kOffSrc + (size_t)kMaxN * sizeof(int32_t));
constexpr size_t kOffHctl = align256(kOffCtl + sizeof(bcgb::DevCtl));
constexpr size_t kOffDummy = align256(kOffHctl + sizeof(bcgb::HostCtl));
constexpr size_t kNeed = align256(kOffDummy + 256);
static_assert(kNeed <= BC_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

// The shared scratch of every bc_run_noalloc call on this device.
__device__ __align__(256) unsigned char g_noalloc_scratch[BC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once.
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

// Input checks on the device (the inputs are device pointers): row_ptr
// starts at 0 and never decreases, neighbour ids and source ids are in range.
// Also writes the work items (one per vertex) and, when sources is null, the
// list 0..n-1. Any violation sets bit 1 of *bad.
__global__ void k_noalloc_prepare(int32_t n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                  const int32_t *__restrict__ sources, int32_t nsrc, int32_t *items,
                                  int32_t *iota, uint32_t *bad) {
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && row_ptr[0] != 0) atomicOr(bad, 1u);
    for (int v = tid; v < n; v += stride) {
        const int a = row_ptr[v], b = row_ptr[v + 1];
        if (b < a) atomicOr(bad, 1u);
        items[v] = v;                 // item_v
        items[kMaxN + v] = a;         // item_beg
        items[2 * kMaxN + v] = b;     // item_end
        items[3 * kMaxN + v] = -1;    // item_slot: no split vertices here
        if (!sources) iota[v] = v;
    }
    const int m2 = row_ptr[n];
    for (int e = tid; e < m2; e += stride)
        if (col[e] < 0 || col[e] >= n) atomicOr(bad, 1u);
    if (sources)
        for (int i = tid; i < nsrc; i += stride)
            if (sources[i] < 0 || sources[i] >= n) atomicOr(bad, 1u);
}

}  // namespace

extern "C" int bc_run_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *sources,
                              int32_t num_sources, double *bc, void *cuda_stream) {
    if (n < 0 || n > kMaxN) return BC_ERR_ARG;
    if (!row_ptr || (n > 0 && (!col || !bc)) || (sources && num_sources < 0)) return BC_ERR_ARG;
    if (sources && num_sources > kMaxN) return BC_ERR_ARG;
    if (n == 0) return BC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return BC_ERR_CUDA;
    const int32_t nsrc = sources ? num_sources : n;

    bcgb::MsParams p{};
    p.n = n;
    p.nitems = n;
    p.nw32 = (n + 31) / 32;
    p.Lcap = kLcap;
    p.row_ptr = row_ptr;
    p.col = col;
    p.col_f = col;  // undirected: the forward pulls over the same arcs
    int32_t *items = reinterpret_cast<int32_t *>(base + kOffItems);
    p.item_v = items;
    p.item_beg = items + kMaxN;
    p.item_end = items + 2 * kMaxN;
    p.item_slot = items + 3 * kMaxN;
    int32_t *dummy = reinterpret_cast<int32_t *>(base + kOffDummy);
    p.slot_first = dummy;  // never read: no item has a slot
    p.slot_nch = dummy;
    p.sigma = reinterpret_cast<uint64_t *>(base + kOffSigma);
    p.S = reinterpret_cast<uint16_t *>(base + kOffS);
    p.s_levels = 2;  // two masked-row buffers by level parity (the backward reads sigma)
    p.wide = reinterpret_cast<uint32_t *>(base + kOffWide);
    p.cval = reinterpret_cast<float *>(base + kOffCval);
    p.F = reinterpret_cast<uint32_t *>(base + kOffF);
    p.ufr = reinterpret_cast<uint32_t *>(base + kOffUfr);
    p.V = reinterpret_cast<uint32_t *>(base + kOffV);
    p.part = reinterpret_cast<uint64_t *>(dummy);
    p.pmask = reinterpret_cast<uint32_t *>(dummy);
    p.cnt = reinterpret_cast<uint32_t *>(dummy);
    p.bc = bc;
    p.ctl = reinterpret_cast<bcgb::DevCtl *>(base + kOffCtl);
    p.hctl = reinterpret_cast<bcgb::HostCtl *>(base + kOffHctl);  // device memory here: nobody polls it
    int32_t *iota = reinterpret_cast<int32_t *>(base + kOffSrc);

    // the scratch keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(p.ctl, 0, sizeof(bcgb::DevCtl), st) != cudaSuccess) return BC_ERR_CUDA;
    if (cudaMemsetAsync(bc, 0, (size_t)n * sizeof(double), st) != cudaSuccess) return BC_ERR_CUDA;
    k_noalloc_prepare<<<64, 256, 0, st>>>(n, row_ptr, col, sources, nsrc, items, iota, &p.ctl->pad[0]);
    uint32_t bad = 0;
    if (cudaMemcpyAsync(&bad, &p.ctl->pad[0], sizeof(bad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BC_ERR_CUDA;
    if (bad) return BC_ERR_ARG;
    const int32_t *src = sources ? sources : iota;

    uint32_t seq = 0;
    for (int32_t b0 = 0; b0 < nsrc; b0 += kB) {
        p.nb = nsrc - b0 < kB ? nsrc - b0 : kB;
        p.seq = ++seq;
        p.sources = src + b0;
        bcgb::ms_launch_init(kW, p, st);
        // forward levels in groups of four; the device flag stops the pass
        struct {
            uint32_t status, fwd_done;
            int32_t nlevels;
        } c = {0, 0, 0};
        int launched = 0;
        while (!c.fwd_done) {
            if (launched > kLcap - 2) return BC_ERR_STATE;  // the kernels always stop before this
            for (int k = 0; k < 4 && launched <= kLcap - 2; ++k) bcgb::ms_launch_forward(kW, p, launched++, st);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&c, p.ctl, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return BC_ERR_CUDA;
        }
        if (c.nlevels < 0) return BC_ERR_UNSUPPORTED;  // deeper than BC_NOALLOC_MAX_LEVELS
        for (int l = c.nlevels; l >= 1; --l) bcgb::ms_launch_backward(kW, p, l, st);
        if (cudaGetLastError() != cudaSuccess) return BC_ERR_CUDA;
    }
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, &p.ctl->status, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BC_ERR_CUDA;
    // a wait for staged row copies that gave up leaves rows incomplete: the
    // result cannot be trusted
    if (status & BC_STATUS_COPY_TIMEOUT) return BC_ERR_TIMEOUT;
    return (status & BC_STATUS_SIGMA_OVERFLOW) ? BC_WARN_SIGMA_OVERFLOW : BC_OK;
}
