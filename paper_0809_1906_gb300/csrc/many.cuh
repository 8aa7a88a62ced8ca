// many.cuh -- descriptors of the many-graph persistent launch (many.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bc_internal.cuh"

namespace bcgb {

struct ManyGraph {
    int32_t n;
    int32_t nitems;    // work items of this graph (> 1: split, partials combined)
    int64_t part_off;  // first partial vector of a split graph in ManyParams::partial
    const int32_t *row_ptr;
    const int32_t *col;
    double *bc;  // the graph's result vector
    // per-source summaries in source (= vertex) order, or null: for source s,
    // sum_v sigma_s(v) (v+1), sum_v (d(s,v)+1) (v+1), sum_v d(s,v) and the
    // number of vertices reached, v over the vertices reachable from s
    uint64_t *h_sigma, *h_dist;
    int64_t *dist_sum, *reach;
};

struct ManyItem {
    int32_t graph;
    int32_t batch_lo, batch_hi;  // source batches [lo, hi) of 32*W sources each
    int32_t part;                // index of this item among its graph's items
};

struct ManyParams {
    int32_t ngraphs, nitems;
    int32_t nmax, nw32max, Lcap;
    const ManyGraph *graphs;
    const ManyItem *items;
    unsigned *queue;    // next item to take
    unsigned *arrive;   // [ngraphs] finished items of each split graph
    unsigned *capped;   // [ngraphs] set when a graph is deeper than Lcap levels
    double *partial;    // partial BC vectors of split graphs
    uint64_t *sigma;    // per-CTA workspaces
    uint16_t *S;        // [2][nmax][B] masked forward rows
    float *cval;        // [2][nmax][B] masked backward rows
    uint32_t *F, *V, *ufr;
    DevCtl *ctl;
};

int many_blocks_per_sm(int W);
void many_launch(int W, const ManyParams &p, int grid, cudaStream_t st);

}  // namespace bcgb
