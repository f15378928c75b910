// Host runtime of the batched step: a batch holds a device table of member
// contexts and advances all of them with one persistent launch per kernel
// kind per step, optionally replayed from a captured CUDA graph.
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cstddef>

#include "tlsph_internal.cuh"

using namespace tlsph;

struct tlsph_batch {
    int capacity = 0;
    cudaStream_t stream = nullptr;  // the caller's stream (ordering)
    cudaStream_t own = nullptr;     // the batch's launches (a non-default stream, as graph capture needs)
    cudaEvent_t start = nullptr;
    void *mem = nullptr;          // BatchHdr followed by capacity BatchSlots
    BatchHdr *hdr = nullptr;
    BatchSlot *slots = nullptr;
    int64_t *blk0 = nullptr;        // capacity first work blocks (device), after the slots
    std::vector<int64_t> blk0_host;
    std::vector<BatchSlot> host;
    std::vector<tlsph_ctx *> members;
    std::vector<int64_t> steps_at;  // each member's step count the table was built for
    int hg = -1;                    // hourglass on/off shared by the members
    int shape[BATCH_KINDS] = { 0, 0, 0 };                 // launch-shape variant per kernel kind
    int grid[2][4] = { { 0, 0, 0, 0 }, { 0, 0, 0, 0 } };   // persistent grids per kernel kind, without / with hourglass
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_hg = -1;
    cudaEvent_t done = nullptr;     // end of the last batch step (members' streams wait on it)
    std::string err;
};

namespace {

int batch_fail(tlsph_batch *b, int code, const std::string &msg)
{
    b->err = msg;
    return code;
}

}  // namespace

extern "C" {

int tlsph_batch_create(int capacity, void *stream, tlsph_batch **out)
{
    if (!out || capacity <= 0 || capacity > (1 << 20)) return TLSPH_ERR_ARG;
    *out = nullptr;
    tlsph_batch *b = new (std::nothrow) tlsph_batch();
    if (!b) return TLSPH_ERR_NOMEM;
    b->capacity = capacity;
    b->stream = static_cast<cudaStream_t>(stream);
    const size_t bytes = 256 + (size_t)capacity * sizeof(BatchSlot) + (size_t)capacity * sizeof(int64_t);
    if (cudaMalloc(&b->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return TLSPH_ERR_NOMEM;
    }
    b->hdr = static_cast<BatchHdr *>(b->mem);
    b->slots = reinterpret_cast<BatchSlot *>(static_cast<char *>(b->mem) + 256);
    b->blk0 = reinterpret_cast<int64_t *>(b->slots + capacity);
    BatchHdr h{ 0, 0, b->blk0 };
    if (cudaMemcpy(b->hdr, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (b->done) cudaEventDestroy(b->done);
        if (b->start) cudaEventDestroy(b->start);
        cudaFree(b->mem);
        delete b;
        return TLSPH_ERR_CUDA;
    }
    *out = b;
    return TLSPH_OK;
}

int tlsph_batch_set(tlsph_batch *b, tlsph_ctx *const *ctxs, int n)
{
    if (!b || n < 0 || (n > 0 && !ctxs)) return TLSPH_ERR_ARG;
    if (n > b->capacity) return batch_fail(b, TLSPH_ERR_ARG, "more contexts than the batch capacity");
    int hg = -1;
    for (int k = 0; k < n; ++k) {
        tlsph_ctx *c = ctxs[k];
        if (!c) return batch_fail(b, TLSPH_ERR_ARG, "NULL context");
        if (c->sticky) return batch_fail(b, TLSPH_ERR_STATE, "a member context holds an error");
        if (c->cfg.precision != TLSPH_PRECISION_MIXED || !c->ell_ok)
            return batch_fail(b, TLSPH_ERR_ARG, "batched stepping needs mixed-precision contexts with sliced-ELL columns");
        const int h = c->cfg.hg_alpha != 0.0 ? 1 : 0;
        if (hg >= 0 && h != hg) return batch_fail(b, TLSPH_ERR_ARG, "members must all use hourglass control or none");
        hg = h;
        for (int m = 0; m < TLSPH_MAX_MATERIALS; ++m)
            if (c->mat_used[m] && !c->mat_set[m]) return batch_fail(b, TLSPH_ERR_STATE, "a member has an unset material");
        for (int m = 0; m < k; ++m)
            if (ctxs[m] == c) return batch_fail(b, TLSPH_ERR_ARG, "a context appears twice");
    }
    cudaError_t e = cudaSuccess;
    // every member ready to step: its own stream idle, half-step quantities current
    for (int k = 0; k < n; ++k) {
        tlsph_ctx *c = ctxs[k];
        e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess && c->need_predict) {
            e = launch_predict(c->s, c->ucur, c->cfg.dt, (c->cfg.flags & TLSPH_FLAG_WALL) != 0, c->steps, c->stream);
            if (e == cudaSuccess) e = mixed_after_predict(c->s, c->dcur, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess) c->need_predict = false;
        }
        if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("member set-up: ") + cudaGetErrorString(e));
    }
    if (b->shape[0] == BATCH_TABLE_VARIANT)       // the pass-1 gather variant reads the members' weight tables
        for (int k = 0; k < n; ++k) {
            const int r = ctx_weight_table(ctxs[k]);
            if (r != TLSPH_OK) return batch_fail(b, r, std::string("member weight table: ") + ctxs[k]->err);
        }
    b->host.resize(n);
    b->members.assign(ctxs, ctxs + n);
    b->steps_at.resize(n);
    int64_t blk = 0;
    b->blk0_host.resize(n);
    for (int k = 0; k < n; ++k) {
        b->host[k] = make_batch_slot(*ctxs[k]);
        b->host[k].blk0 = blk;
        b->blk0_host[k] = blk;
        blk += (ctxs[k]->N + 127) / 128;
        b->steps_at[k] = ctxs[k]->steps;
    }
    BatchHdr h{ n, blk, b->blk0 };
    e = cudaStreamSynchronize(b->own);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(b->slots, b->host.data(), (size_t)n * sizeof(BatchSlot), cudaMemcpyHostToDevice, b->own);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(b->blk0, b->blk0_host.data(), (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, b->own);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->hdr, &h, sizeof h, cudaMemcpyHostToDevice, b->own);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->own);
    if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    if (hg >= 0) b->hg = hg;
    return TLSPH_OK;
}

int tlsph_batch_step(tlsph_batch *b, int nsteps, int use_graph)
{
    if (!b || nsteps < 0) return TLSPH_ERR_ARG;
    const int n = (int)b->members.size();
    if (n == 0 || nsteps == 0) return TLSPH_OK;
    for (int k = 0; k < n; ++k) {
        tlsph_ctx *c = b->members[k];
        if (c->sticky) return batch_fail(b, TLSPH_ERR_STATE, "a member context holds an error");
        if (c->steps != b->steps_at[k] || c->need_predict)
            return batch_fail(b, TLSPH_ERR_STATE, "a member was changed outside the batch: call tlsph_batch_set again");
        if (b->shape[0] == BATCH_TABLE_VARIANT && (!c->s.w1t || c->s.w1t != b->host[k].s.w1t))
            return batch_fail(b, TLSPH_ERR_STATE, "a member's weight table was released: call tlsph_batch_set again");
    }
    const bool hg = b->hg == 1;
    int *grid = b->grid[hg ? 1 : 0];
    if (grid[0] == 0) batch_grid(hg, b->shape, grid);
    // the batch's work follows everything already queued on the caller's stream
    cudaError_t e = cudaEventRecord(b->start, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->own, b->start, 0);
    if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("batch order: ") + cudaGetErrorString(e));
    if (use_graph) {
        if (!b->exec || b->graph_hg != b->hg) {
            if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
            if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
            e = cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = launch_batch_step(b->hdr, b->slots, b->capacity, hg, b->shape, grid, b->own);
                e = cudaStreamEndCapture(b->own, &b->graph);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return batch_fail(b, TLSPH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            }
            b->graph_hg = b->hg;
        }
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = cudaGraphLaunch(b->exec, b->own);
    } else {
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
            e = launch_batch_step(b->hdr, b->slots, b->capacity, hg, b->shape, grid, b->own);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->own);
    // later work on the caller's stream and on each member's own stream is ordered after the batch
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->done, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->members[k]->stream, b->done, 0);
    if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
    // the members' host-side view follows the device slots
    for (int k = 0; k < n; ++k) {
        tlsph_ctx *c = b->members[k];
        if (nsteps & 1) {
            c->ucur ^= 1;
            c->dcur ^= 1;
        }
        c->steps += nsteps;
        b->steps_at[k] = c->steps;
    }
    return TLSPH_OK;
}

int tlsph_batch_sync(tlsph_batch *b)
{
    if (!b) return TLSPH_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(b->own);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? TLSPH_OK : batch_fail(b, TLSPH_ERR_CUDA, cudaGetErrorString(e));
}

const char *tlsph_batch_last_error(const tlsph_batch *b) { return b ? b->err.c_str() : ""; }

int tlsph_batch_set_shape(tlsph_batch *b, const int32_t *shape, int n)
{
    if (!b || !shape || n != BATCH_KINDS) return TLSPH_ERR_ARG;
    for (int k = 0; k < BATCH_KINDS; ++k)
        if (shape[k] < 0 || shape[k] >= BATCH_VARIANTS[k])
            return batch_fail(b, TLSPH_ERR_ARG, "launch-shape variant out of range for kernel kind " + std::to_string(k));
    bool same = true;
    for (int k = 0; k < BATCH_KINDS; ++k) same &= b->shape[k] == shape[k];
    if (same) return TLSPH_OK;
    // the launches in flight use the old kernels and grids: finish them before replacing the graph
    cudaError_t e = cudaStreamSynchronize(b->own);
    if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("set_shape: ") + cudaGetErrorString(e));
    if (shape[0] == BATCH_TABLE_VARIANT) {
        // the members' weight tables, and their pointers patched into the device slots (the rest of a
        // slot carries state the device advances)
        for (size_t k = 0; k < b->members.size(); ++k) {
            tlsph_ctx *c = b->members[k];
            const int r = ctx_weight_table(c);
            if (r != TLSPH_OK) return batch_fail(b, r, std::string("member weight table: ") + c->err);
            b->host[k].s.w1t = c->s.w1t;
            b->host[k].s.w1t_off = c->s.w1t_off;
            static_assert(offsetof(DevState, w1t_off) == offsetof(DevState, w1t) + sizeof(void *),
                          "the two table pointers are adjacent");
            e = cudaMemcpyAsync(reinterpret_cast<char *>(b->slots + k) + offsetof(BatchSlot, s) + offsetof(DevState, w1t),
                                &b->host[k].s.w1t, 2 * sizeof(void *), cudaMemcpyHostToDevice, b->own);
            if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("set_shape: ") + cudaGetErrorString(e));
        }
        e = cudaStreamSynchronize(b->own);
        if (e != cudaSuccess) return batch_fail(b, TLSPH_ERR_CUDA, std::string("set_shape: ") + cudaGetErrorString(e));
    }
    for (int k = 0; k < BATCH_KINDS; ++k) b->shape[k] = shape[k];
    for (auto &g : b->grid)
        for (int &x : g) x = 0;             // recomputed for the new kernels at the next step
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_hg = -1;
    return TLSPH_OK;
}

int tlsph_batch_get_shape(const tlsph_batch *b, int32_t *shape, int32_t *variants, int n)
{
    if (!b || n != BATCH_KINDS) return TLSPH_ERR_ARG;
    for (int k = 0; k < BATCH_KINDS; ++k) {
        if (shape) shape[k] = b->shape[k];
        if (variants) variants[k] = BATCH_VARIANTS[k];
    }
    return TLSPH_OK;
}

int tlsph_batch_destroy(tlsph_batch *b)
{
    if (!b) return TLSPH_ERR_ARG;
    cudaStreamSynchronize(b->own);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->mem) cudaFree(b->mem);
    if (b->done) cudaEventDestroy(b->done);
    if (b->start) cudaEventDestroy(b->start);
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
    return TLSPH_OK;
}

}  // extern "C"
