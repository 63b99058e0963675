// noalloc.cu -- one neighbour level for callers that cannot allocate device memory.
//
// paces_expand_noalloc runs the same level kernels as paces_set_state with
// m_init = 1 (expansion through H's moves, hash de-duplication with
// first-occurrence winners, compaction), but every piece of working memory it
// needs -- model tables, counters, the hash table, candidate slots and winner
// masks -- lives in one file-scope device array of fixed size.  The caller
// passes the input keys and the output buffer; the call performs no cudaMalloc,
// cudaMallocAsync, cudaFree or allocation through any library.
#include <cstring>
#include <mutex>
#include <string>

#include "paces.h"
#include "runtime.h"

namespace paces {
namespace {

static_assert(PACES_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch alignment");

// Shared by every call in the process on this device; contents persist between
// calls and are re-initialised by each call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PACES_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never dereferenced).
cudaError_t scratch_address(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace paces

using namespace paces;

static paces_status need_bytes(const paces_params* params, int64_t n_in, int64_t max_out, int64_t* bytes)
{
    if (!bytes || n_in < 1 || max_out < n_in) return PACES_ERR_INVALID;
    paces_layout L;
    paces_status s = plan_layout_internal(params, &L);
    if (s) return s;
    DevModel* M = new DevModel();
    s = fill_model(params, L, M);
    int D = M->D, W = L.words;
    delete M;
    if (s) return s;
    int64_t rows = std::min<int64_t>(max_out, n_in * (int64_t)(D + 1));
    int64_t slots = 2 * rows + 1;
    size_t sw = W == 1 ? 2 : (W <= 3 ? 4 : 6);
    size_t need = up256(sizeof(DevModel)) + up256(sizeof(Counters)) + 2 * up256(4 * kMaxChunkBlocks) +
                  up256((size_t)slots * sw * 8) + up256((size_t)n_in * D * 4) + up256((size_t)n_in * 8) +
                  up256((size_t)rows * sizeof(double2)) + up256((size_t)rows * 4);
    *bytes = (int64_t)need;
    return PACES_OK;
}

extern "C" paces_status paces_expand_noalloc(const paces_params* params, const uint64_t* keys_in, int64_t n_in,
                                             uint64_t* keys_out, int64_t max_out, int64_t* n_out, void* stream)
{
    if (!params || !keys_in || !keys_out || !n_out || n_in < 1 || max_out < n_in) return PACES_ERR_INVALID;
    paces_layout L;
    paces_status s = plan_layout_internal(params, &L);
    if (s) return s;
    DevModel* M = new DevModel();          // host memory only
    s = fill_model(params, L, M);
    if (s) {
        delete M;
        return s;
    }
    const int W = L.words, D = M->D;
    // every input key needs 8 bytes of winner mask in the scratch array, so a
    // larger n_in cannot fit; rejecting it first keeps the size products below
    // far from overflow
    if (n_in > (int64_t)(PACES_NOALLOC_SCRATCH_BYTES / 8) || n_in >= (int64_t)kCand / (D + 1)) {
        delete M;
        return PACES_ERR_CAPACITY;
    }
    int64_t need = 0;
    need_bytes(params, n_in, max_out, &need);
    if (need > (int64_t)PACES_NOALLOC_SCRATCH_BYTES || n_in * (int64_t)D >= (int64_t)kCand) {
        delete M;
        return PACES_ERR_CAPACITY;         // beyond the fixed scratch: use paces_set_state instead
    }
    int dev = 0, sms = 0;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        scratch_address(dev, &base) != cudaSuccess) {
        delete M;
        return PACES_ERR_CUDA;
    }
    int64_t rows = std::min<int64_t>(max_out, n_in * (int64_t)(D + 1));
    uint64_t slots = 2ull * (uint64_t)rows + 1;
    size_t sw = W == 1 ? 2 : (W <= 3 ? 4 : 6);

    Bufs b{};
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += up256(bytes);
        return (void*)p;
    };
    b.model = (const DevModel*)carve(sizeof(DevModel));
    b.ctr = (Counters*)carve(sizeof(Counters));
    b.blk_cnt = (uint32_t*)carve(4 * kMaxChunkBlocks);
    b.blk_off = (uint32_t*)carve(4 * kMaxChunkBlocks);
    b.table[0] = (uint64_t*)carve((size_t)slots * sw * 8);
    b.cand_slot = (uint32_t*)carve((size_t)n_in * D * 4);
    b.masks = (uint64_t*)carve((size_t)n_in * 8);
    b.V[1] = (double2*)carve((size_t)rows * sizeof(double2));
    b.V[0] = b.V[1];                       // no previous state: rescue is off
    b.meta[0] = (uint32_t*)carve((size_t)rows * 4);
    b.keys[0] = keys_out;
    b.table_slots = slots;
    b.cap_rows = (uint32_t)rows;
    b.cand_cap = (uint64_t)n_in * D;
    b.W = W;
    b.D = D;
    b.P = M->P;
    b.N = params->n_sites;
    b.G = std::min(kMaxChunkBlocks, sms * 4);
    b.grid = sms * 8;

    Counters c;
    std::memset(&c, 0, sizeof(c));
    c.q = c.q_in = c.kept = (uint32_t)n_in;
    c.level_off[1] = (uint32_t)n_in;
    c.nlevels = 1;
    cudaError_t e = cudaMemcpyAsync((void*)b.model, M, sizeof(DevModel), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.ctr, &c, sizeof(Counters), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.table[0], 0xFF, (size_t)slots * sw * 8, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(keys_out, keys_in, (size_t)n_in * W * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        launch_meta_from_keys(b, 0, (uint32_t)n_in, st);
        launch_insert_rows(b, 0, (uint32_t)n_in, st);
        launch_level(b, 0, 0, -1, 0, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, b.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    delete M;
    if (e != cudaSuccess) return PACES_ERR_CUDA;
    if (c.err == kErrRows || c.err == kErrProbe || c.err == kErrCand) return PACES_ERR_CAPACITY;
    if (c.err) return PACES_ERR_CUDA;
    *n_out = (int64_t)c.q;
    return PACES_OK;
}
