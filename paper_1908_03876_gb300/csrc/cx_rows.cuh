// cx_rows.cuh -- the warp-specialised row-window pipeline shared by the
// forward and adjoint row-window kernels.
//
// A block is NT compute threads (one node of a row segment each) plus one
// producer warp.  Lane 0 of the producer issues, per row segment, the bulk
// asynchronous copies (cp.async.bulk) of the segment's staged data into one of
// ROWS_STAGES shared-memory stages; the copies complete on that stage's "full"
// mbarrier.  Compute warps wait on "full", compute their nodes from the stage,
// and release it with one arrival per warp on the stage's "empty" mbarrier;
// the producer reuses a stage once every compute warp has released it.  No
// block-wide barrier runs inside the loop, so a warp that finishes a segment
// early moves on to the next staged one instead of waiting for the slowest
// warp, and the producer keeps up to ROWS_STAGES - 1 segments in flight.
//
// Every wait is bounded in time (MBAR_WAIT_NS): a wait that runs out sets a
// block-local abort flag and ST_TIMEOUT in the status word; the other threads
// then leave at their next wait, and the producer, before leaving, waits
// (again bounded) for the copies it issued to land, so no copy writes shared
// memory after the block has left.
#pragma once

#include "cx_device.cuh"

namespace cx {

constexpr int ROWS_STAGES = 3;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// dynamic shared memory of a pipeline with stages of sv values of T
template <typename T> constexpr size_t rows_pipe_smem(int sv) {
    return (size_t)ROWS_STAGES * sv * sizeof(T) + 2 * ROWS_STAGES * sizeof(uint64_t) + 16;
}

template <typename T, int NT> struct RowsPipe {
    static constexpr int S = ROWS_STAGES;
    T* st;                        // stage 0; stage b at st + b * sv
    int sv;                       // values of T per stage
    uint64_t* full;               // [S] copies of the stage landed
    uint64_t* empty;              // [S] every compute warp released the stage
    volatile int* abort_flag;     // a bounded wait ran out somewhere in the block

    __device__ __forceinline__ RowsPipe(unsigned char* smem, int sv_) : sv(sv_) {
        st = reinterpret_cast<T*>(smem);
        full = reinterpret_cast<uint64_t*>(st + S * sv_);
        empty = full + S;
        abort_flag = reinterpret_cast<volatile int*>(empty + S);
    }
    __device__ __forceinline__ T* stage(int b) const { return st + b * sv; }

    // thread 0, before the block-wide barrier that publishes it
    __device__ __forceinline__ void init() {
        if (threadIdx.x == 0) {
            for (int i = 0; i < S; ++i) {
                mbar_init(&full[i], 1);
                mbar_init(&empty[i], NT / 32);
            }
            *abort_flag = 0;
            mbar_init_fence();
        }
    }

    // Producer (lane 0 of the warp after the compute threads): issue(y, x0,
    // stage, full_bar) for each of the block's row segments in order.
    template <typename Issue> __device__ __forceinline__ void produce(const CxConst& C, int* status, Issue issue) {
        if (threadIdx.x != NT) return;
        ChunkIter<NT> it(C);
        int s = 0;
        bool ok = true;
        for (; it.valid(); it.next(), ++s) {
            const int b = s % S;
            if (s >= S) { // stage b held segment s - S: wait until every compute warp released it
                ok = mbar_wait(&empty[b], (unsigned)(s / S - 1) & 1u);
                if (!ok) break;
            }
            if (*abort_flag) break;
            issue(it.y, it.seg * NT, stage(b), &full[b]);
        }
        if (!ok) {
            *abort_flag = 1;
            if (status) atomicOr(status, ST_TIMEOUT);
        }
        // the last (up to S) issued segments may still be landing
        for (int j = (s > S ? s - S : 0); j < s; ++j) mbar_wait(&full[j % S], (unsigned)(j / S) & 1u);
    }

    // Compute threads: ctrl(node, stage) stages this thread's own per-node
    // values by cp.async (S - 1 segments ahead, into stages this thread has
    // finished with); compute(node, stage) runs the node body.
    // The node description of the next segment (its solid and mask bytes come
    // from global memory) is read one segment ahead, so those loads overlap
    // the current segment's work.
    template <typename Ctrl, typename Compute>
    __device__ __forceinline__ void consume(const CxConst& C, int* status, Ctrl ctrl, Compute compute) {
        ChunkIter<NT> it(C), ahead(C);
        for (int j = 0; j < S - 1; ++j) {
            if (ahead.valid()) ctrl(ahead.node(C), stage(j));
            cp_async_commit();
            ahead.next();
        }
        unsigned fl = it.valid() ? it.flags(C) : 0u;
        for (int s = 0; it.valid(); ++s) {
            const int b = s % S;
            const NodeIdx cur = it.node_from(C, fl);
            if (ahead.valid()) ctrl(ahead.node(C), stage((s + S - 1) % S));
            cp_async_commit();
            ahead.next();
            it.next();
            fl = it.valid() ? it.flags(C) : 0u; // the next segment's bytes, used in the next iteration
            cp_async_wait<S - 1>(); // this thread's own copies for segment s
            const bool ok = !*abort_flag && mbar_wait(&full[b], (unsigned)(s / S) & 1u);
            if (ok) compute(cur, stage(b));
            __syncwarp();
            if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[b]);
            if (!ok) {
                *abort_flag = 1;
                if ((threadIdx.x & 31) == 0 && status) atomicOr(status, ST_TIMEOUT);
                break;
            }
        }
        cp_async_wait<0>();
    }
};

} // namespace cx
