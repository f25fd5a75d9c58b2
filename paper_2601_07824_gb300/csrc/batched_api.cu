// batched_api.cu -- hadamag_sre_batched: host planning, autotuning and launch of batched.cu.
//
// The autotuner picks, per set of state sizes (and gradient on/off) and per large state size N,
// the number of X-strings A that a pass-1 task covers (the x-batch: 8, 4 or 2), by timing a
// launch of up to two states of that size per candidate on the first uncaptured call, and
// caches the choice.  The pass-1 width
// (10 bits) and the small/large split (N <= 14: one-pass chunk items) are fixed by the kernels.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "batched.h"
#include "ctx.h"

using namespace hm;

namespace {

// Partial-gradient buffer slots of the large states, taken in turn.  The large states run one
// after another in the static phase, and at most two adjacent ones are in flight at a time
// (a CTA starts state k + 1 only after its own tasks of state k, and state k's pass 2 needs
// every CTA's pass 1 of state k), so state k's pass 3 rarely waits for state k - 2's finalize.
constexpr int kPartSlots = 2;

struct Plan {
    std::vector<BatchState> st;
    int64_t total = 0;
    size_t scratch_bytes = 0, gsmall_bytes = 0;
    int n_large = 0;
    int64_t dimmax = 1;
};

// Builds the state table (offsets into the context buffers are filled in later).
Plan make_plan(int count, const void* const* psi, const int* N, void* const* grad, const int* A_of_N, bool fwd,
               int grid) {
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const bool lx = N[x] >= 15, ly = N[y] >= 15;
        if (lx != ly) return lx;  // large states (the static phase) first, then small ones
        return N[x] > N[y];       // largest first
    });
    Plan p;
    for (int i : order) {
        BatchState s{};
        s.psi = reinterpret_cast<const float2*>(psi[i]);
        s.grad = grad ? reinterpret_cast<float2*>(grad[i]) : nullptr;
        s.N = N[i];
        s.task_begin = p.total;  // small states: tickets (large states run a static schedule)
        s.out_idx = i;
        s.fwd = fwd ? 1 : 0;
        const int64_t dim = int64_t(1) << s.N;
        if (s.N <= 14) {
            // X-string chunks of about 2^23 Pauli strings each (N = 14: 32, 13: 8, 12: 2, else
            // 1), at most one per S_2 slot of the state
            s.kind = 0;
            s.n_chunks = (int)std::min<int64_t>(2 * kS2Lanes, std::max<int64_t>(1, (dim * dim) >> 23));
            if (!fwd) p.gsmall_bytes += (size_t)s.n_chunks * (256 >> (s.N - 6)) * dim * sizeof(float2);
            p.total += s.n_chunks + (s.n_chunks > 1 ? 1 : 0);
        } else {
            s.kind = 1;
            const int M = s.N - 11;
            s.A = A_of_N[s.N];
            s.U = 8 / s.A;
            s.n_batches = dim / s.A;
            // 2 units per pass-1 warp, 1 column tile per pass-2 task (larger tasks leave too few
            // per pipeline stage at N <= 18; measured slower)
            const int tiles = 1024 >> (13 - M);
            s.UPW = 2;
            s.TPT = 1;
            s.p1 = (1 << M) / (s.U * s.UPW);
            s.p2 = s.A * tiles / s.TPT;
            s.p3 = s.A * ((1 << M) / 16);
            // stages between the passes of a batch (the single-state rule: N = 15: 15, 16: 8,
            // 17: 4, 18: 2 at A = 8 and two CTAs per SM), ring of 2 lag + 1 slots
            s.lag = pipeline_lag((int64_t)s.p1 + s.p2 + (fwd ? 0 : s.p3), grid, 2,
                                 (size_t)s.A * (size_t)(dim / 2) * sizeof(float2), (size_t)96 << 20);
            s.R = 2 * s.lag + 1;
            if (fwd) {
                s.n_stage_tasks = (s.n_batches + s.lag) * ((int64_t)s.p1 + s.p2);
                s.n_fin = 1;
            } else {
                s.n_stage_tasks = (s.n_batches + 2 * s.lag) * ((int64_t)s.p1 + s.p2 + s.p3);
                s.n_fin = (int)std::max<int64_t>(1, dim / 2048);
            }
            p.scratch_bytes += (size_t)s.R * s.A * (size_t)(dim / 2) * sizeof(float2);
            p.n_large++;
            p.dimmax = std::max(p.dimmax, dim);
        }
        p.st.push_back(s);
    }
    return p;
}

struct TuneKey {
    std::string key;
};

std::string tune_key(int count, const int* N, int want_grad) {
    std::vector<int> v(N, N + count);
    std::sort(v.begin(), v.end());
    std::string k = want_grad ? "g" : "f";
    for (int n : v) k += "," + std::to_string(n);
    return k;
}

// x-batch per state size (index N; only 15..18 are read)
struct XBatch {
    int A[19];
};

std::map<std::string, XBatch>& tune_cache() {
    static std::map<std::string, XBatch> m;
    return m;
}

hadamag_status run(hadamag_ctx_t c, int count, const void* const* psi, const int* N, int want_grad,
                   void* const* grad, double* m2, cudaStream_t st, const int* A_of_N) {
    hadamag_status s;
    cudaError_t e;
    int grid = 0;
    if ((e = batched_max_grid(c->sm_count, &grid)) != cudaSuccess) return cuda_fail(c, e, "occupancy");
    Plan p = make_plan(count, psi, N, want_grad ? grad : nullptr, A_of_N, !want_grad, grid);
    const int ns = (int)p.st.size();
    // one device allocation carved into: table | counters | s2 | ticket (buffers below separately)
    const size_t table_bytes = (size_t)ns * sizeof(BatchState);
    const size_t ctr_bytes = (size_t)ns * 256 * sizeof(unsigned);
    const size_t s2_bytes = (size_t)ns * 2 * kS2Lanes * sizeof(double);
    const size_t meta_bytes = table_bytes + ctr_bytes + s2_bytes + 256;
    if ((s = ensure_buf(c, c->batch_meta, meta_bytes))) return s;
    if ((s = ensure_buf(c, c->scratch, std::max<size_t>(p.scratch_bytes, 256)))) return s;
    if ((s = ensure_buf(c, c->batch_sums, std::max<size_t>(p.gsmall_bytes, 256)))) return s;
    // partial-gradient buffer slots, taken in turn (slot = large-state index mod slots)
    const size_t slot_bytes = (size_t)grid * p.dimmax * sizeof(float2);
    int slots = 0;
    if (p.n_large && want_grad) {
        slots = std::min(p.n_large, kPartSlots);
    }
    const size_t gpart_bytes = slots ? (size_t)slots * slot_bytes : 256;
    if ((s = ensure_buf(c, c->grad_acc, gpart_bytes))) return s;
    if (c->host_table_bytes < table_bytes) {
        if (c->host_table) cudaFreeHost(c->host_table);
        c->host_table = nullptr;
        c->host_table_bytes = 0;
        if (cudaMallocHost(&c->host_table, table_bytes) != cudaSuccess) return fail(c, HADAMAG_ERR_OOM, "pinned table");
        c->host_table_bytes = table_bytes;
    }
    char* meta = (char*)c->batch_meta.ptr;
    unsigned* ctr = (unsigned*)(meta + table_bytes);
    double* s2 = (double*)(meta + table_bytes + ctr_bytes);
    unsigned long long* ticket = (unsigned long long*)(meta + table_bytes + ctr_bytes + s2_bytes);
    size_t soff = 0, goff = 0;
    std::vector<const unsigned*> slot_fin(slots > 0 ? slots : 1, nullptr);
    std::vector<unsigned> slot_nfin(slots > 0 ? slots : 1, 0u);
    int li = 0;  // large-state index
    for (int k = 0; k < ns; ++k) {
        BatchState& b = p.st[k];
        b.ctr = ctr + (size_t)k * 256;
        b.fin = b.ctr + 192;
        b.s2 = s2 + 2 * kS2Lanes * k;
        if (b.kind == 0) {
            if (want_grad) {
                b.gsmall = (float2*)((char*)c->batch_sums.ptr + goff);
                goff += (size_t)b.n_chunks * (256 >> (b.N - 6)) * ((size_t)1 << b.N) * sizeof(float2);
            }
        } else {
            b.scratch = (float2*)((char*)c->scratch.ptr + soff);
            soff += (size_t)b.R * b.A * ((size_t)1 << (b.N - 1)) * sizeof(float2);
            if (slots) {
                const int sl = li % slots;
                b.gpart = (float2*)((char*)c->grad_acc.ptr + (size_t)sl * slot_bytes);
                b.prev_fin = slot_fin[sl];
                b.prev_nfin = slot_nfin[sl];
                slot_fin[sl] = b.fin;
                slot_nfin[sl] = (unsigned)b.n_fin;
            }
            ++li;
        }
    }
    std::memcpy(c->host_table, p.st.data(), table_bytes);
    if ((e = cudaMemcpyAsync(meta, c->host_table, table_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, e, "copy table");
    if ((e = cudaMemsetAsync(ctr, 0, ctr_bytes + s2_bytes + 256, st)) != cudaSuccess) return cuda_fail(c, e, "memset");
    if (p.gsmall_bytes && (e = cudaMemsetAsync(c->batch_sums.ptr, 0, p.gsmall_bytes, st)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    if (p.n_large && want_grad && (e = cudaMemsetAsync(c->grad_acc.ptr, 0, gpart_bytes, st)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    BatchedParams B{};
    B.states = (const BatchState*)meta;
    B.n_states = ns;
    B.n_large = p.n_large;
    B.total = p.total;
    B.ticket = ticket;
    B.nparts = grid;
    B.m2_out = m2;
    B.ctl = G3Ctl{(int*)c->status.ptr, c->spin_limit, c->wait_bias};
    e = launch_batched(B, !want_grad, grid, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "batched_kernel");
    return HADAMAG_OK;
}

}  // namespace

extern "C" hadamag_status hadamag_sre_batched(hadamag_ctx_t c, int count, const void* const* psi, const int* N,
                                              int want_grad, void* const* grad, double* m2, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (count < 1 || !psi || !N || !m2 || (want_grad && !grad))
        return fail(c, HADAMAG_ERR_INVALID_ARG, "bad batch arguments");
    for (int i = 0; i < count; ++i) {
        if (N[i] < 10 || N[i] > 18) return fail(c, HADAMAG_ERR_INVALID_ARG, "batched states need 10 <= N <= 18");
        if (!aligned16(psi[i]) || (want_grad && !aligned16(grad[i])))
            return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer in batch");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    c->last_error[0] = 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if ((e = cudaMemsetAsync(c->status.ptr, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "memset");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(c, e, "capture query");
    const std::string key = tune_key(count, N, want_grad);
    auto it = tune_cache().find(key);
    XBatch xb;
    for (int& a : xb.A) a = 8;
    if (it != tune_cache().end()) {
        xb = it->second;
    } else if (cap == cudaStreamCaptureStatusNone && c->autotune) {
        // per large size N: time a launch of (up to) two of its states for each candidate x-batch,
        // keep the fastest (the best A differs between sizes: the rows shared at A = 8 against
        // more, smaller pass-1 tasks at A = 2)
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return fail(c, HADAMAG_ERR_CUDA, "events");
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(c, HADAMAG_ERR_CUDA, "events"); }
        hadamag_status s = HADAMAG_OK;
        for (int n = 15; n <= 18 && !s; ++n) {
            std::vector<const void*> sp;
            std::vector<void*> sg;
            std::vector<int> sn;
            for (int i = 0; i < count && sp.size() < 2; ++i)
                if (N[i] == n) { sp.push_back(psi[i]); sg.push_back(want_grad ? grad[i] : nullptr); sn.push_back(n); }
            if (sp.empty()) continue;
            float best = 1e30f;
            for (int cand : {8, 4, 2}) {
                XBatch t = xb;
                t.A[n] = cand;
                cudaEventRecord(e0, st);
                if ((s = run(c, (int)sp.size(), sp.data(), sn.data(), want_grad, sg.data(), m2, st, t.A))) break;
                cudaEventRecord(e1, st);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { s = cuda_fail(c, e, "tune sync"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; xb.A[n] = cand; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s) return s;
        tune_cache()[key] = xb;
    }
    return run(c, count, psi, N, want_grad, grad, m2, st, xb.A);
}

extern "C" hadamag_status hadamag_batched_status(hadamag_ctx_t c, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return finish(c, nullptr, 0, st);
}
