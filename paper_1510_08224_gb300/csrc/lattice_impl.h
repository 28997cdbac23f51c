// Host-side state of one lattice, shared by lbm_api.cu and lbm_batch.cu.
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>
#include <string>
#include <vector>

#include "nomrt_internal.h"

struct lbm_batch;
struct lbm_lattice;

namespace nomrt {

// Removes h from batch b (lbm_destroy of a lattice that is still batched).
void batch_detach(lbm_batch *b, lbm_lattice *h);

// Device layout of one lattice, all offsets from the block base.
struct Layout {
    int nq = 14;                // population planes per buffer: 9 + 5 or 9 + 9
    int pitch = 0;
    size_t plane = 0;           // elements per plane
    size_t pop_bytes = 0;       // one buffer
    size_t off_pop[2] = {0, 0};
    size_t off_mask = 0, off_flags = 0, off_walls = 0, off_snap = 0, off_stage = 0, off_part = 0, off_res = 0,
           off_status = 0, off_nee_dir = 0, off_nee = 0;
    int stage_rows = 0;
    size_t total = 0;
};


}  // namespace nomrt

struct lbm_lattice {
    int nx = 0, ny = 0, px = 0, py = 0, storage = 0, n_walls = 0;
    cudaStream_t stream = nullptr;
    char *mem = nullptr;
    bool owns_mem = false;
    nomrt::Layout lay;
    nomrt::KParams kp;
    int cur = 0;
    int have_snap = 0;
    int64_t fluid = 0;
    int64_t steps = 0;
    int across_x = 0, across_y = 0;  // fluid cells of the middle row / column (lbm_nusselt's default L)
    std::string err;
    const nomrt::Launchers *L = nullptr;
    lbm_batch *batch = nullptr;  // the batch that steps this lattice, if any
    // lbm_step replays graphs of kGraphSteps and kGraphShort steps from buffer 0 once the
    // current step kernel has run directly; reset when the kernel choice changes
    cudaGraphExec_t graph = nullptr;        // kGraphSteps steps
    cudaGraphExec_t graph_short = nullptr;  // kGraphShort steps
    cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on (any stream can launch it)
    int graph_variant = -1, graph_config = -1;
    bool graph_off = false;       // capture failed or the stream cannot be captured
    bool direct_done = false;     // the current kernel choice has run at least once directly

    double *stage() const { return reinterpret_cast<double *>(mem + lay.off_stage); }
    double *partials() const { return reinterpret_cast<double *>(mem + lay.off_part); }
    double *result() const { return reinterpret_cast<double *>(mem + lay.off_res); }
    double *snap() const { return reinterpret_cast<double *>(mem + lay.off_snap); }
};
