// relabel.cu -- a vertex numbering with locality, computed from the CSR alone
// (host code), and the device gather that maps ids through it.
//
// The weighted sweep walks one source's distance buckets per CTA, each
// relaxation a random 8-byte access into that source's per-vertex state. When
// vertices that are close in the graph are also close in memory, one 32-byte
// sector serves several of the accesses a bucket makes, and fewer sectors go
// to DRAM.
//
// The numbering comes from multilevel heavy-edge matching, the coarsening
// step of multilevel graph partitioners. Level 0 is the graph, every edge of
// weight 1. A level visits its nodes in id order; each node not yet matched is
// matched with the unmatched neighbour joined to it by the heaviest edge (the
// first such neighbour in adjacency order). Each matched pair, and each node
// left alone, becomes one node of the next level, numbered in visit order. The
// next level's edge weights are the numbers of edges joining its nodes'
// members. Coarsening stops at one node, or once a level shrinks the graph by
// less than one sixteenth. Vertices are then numbered by their ancestor at the
// top level, then at the level below it, and so on down, with their own ids
// last. Each sector of four consecutive ids then holds, as a rule, the two
// matched pairs that the second level merged, and longer runs of ids hold the
// larger clusters of the levels above.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "weighted.cuh"

namespace bcgb {

void locality_order(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *perm) {
    for (int32_t v = 0; v < n; ++v) perm[v] = v;
    if (n < 2) return;
    // the current level as a weighted CSR
    std::vector<int64_t> xadj(row_ptr, row_ptr + n + 1);
    std::vector<int32_t> adj(col, col + row_ptr[n]);
    std::vector<int32_t> wt(adj.size(), 1);
    std::vector<std::vector<int32_t>> parent;  // parent[k][u]: the level-(k+1) node holding level-k node u
    int32_t m = n;
    while (m > 1 && parent.size() < 64) {
        std::vector<int32_t> match((size_t)m, -1);
        for (int32_t u = 0; u < m; ++u) {
            if (match[u] >= 0) continue;
            int32_t best = -1, bw = 0;
            for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
                const int32_t v = adj[(size_t)e];
                if (v != u && match[v] < 0 && wt[(size_t)e] > bw) {
                    best = v;
                    bw = wt[(size_t)e];
                }
            }
            match[u] = best >= 0 ? best : u;
            if (best >= 0) match[best] = u;
        }
        std::vector<int32_t> cid((size_t)m, -1);
        std::vector<int32_t> first, second;  // members of each next-level node (second: -1 when alone)
        for (int32_t u = 0; u < m; ++u)
            if (cid[u] < 0) {
                const int32_t c = (int32_t)first.size();
                cid[u] = c;
                cid[match[u]] = c;
                first.push_back(u);
                second.push_back(match[u] != u ? match[u] : -1);
            }
        const int32_t c = (int32_t)first.size();
        if (c == m) break;  // nothing matched
        // the next level's edges: each node's members' edges, merged by head
        std::vector<int64_t> nx((size_t)c + 1, 0);
        std::vector<int32_t> na, nw;
        na.reserve(adj.size());
        nw.reserve(adj.size());
        std::vector<int64_t> mark((size_t)c, -1);  // position of a head in the row being built
        for (int32_t x = 0; x < c; ++x) {
            const int64_t row0 = (int64_t)na.size();
            for (int32_t u : {first[x], second[x]}) {
                if (u < 0) continue;
                for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
                    const int32_t y = cid[adj[(size_t)e]];
                    if (y == x) continue;
                    if (mark[y] >= row0) {
                        nw[(size_t)mark[y]] += wt[(size_t)e];
                    } else {
                        mark[y] = (int64_t)na.size();
                        na.push_back(y);
                        nw.push_back(wt[(size_t)e]);
                    }
                }
            }
            nx[(size_t)x + 1] = (int64_t)na.size();
        }
        parent.push_back(std::move(cid));
        const bool slow = c > m - m / 16;
        xadj.swap(nx);
        adj.swap(na);
        wt.swap(nw);
        m = c;
        if (slow) break;
    }
    // top-down numbering: a level's nodes ordered by their parent's position,
    // then by their own id
    std::vector<int32_t> pos((size_t)m);
    for (int32_t x = 0; x < m; ++x) pos[x] = x;
    for (size_t k = parent.size(); k-- > 0;) {
        const std::vector<int32_t> &pk = parent[k];
        const int32_t mk = (int32_t)pk.size();
        std::vector<int32_t> start(pos.size() + 1, 0);
        for (int32_t u = 0; u < mk; ++u) ++start[(size_t)pos[pk[u]] + 1];
        for (size_t i = 1; i < start.size(); ++i) start[i] += start[i - 1];
        std::vector<int32_t> np((size_t)mk);
        for (int32_t u = 0; u < mk; ++u) np[u] = start[pos[pk[u]]]++;
        pos.swap(np);
    }
    for (int32_t v = 0; v < n; ++v) perm[v] = pos[v];
}

namespace {
__global__ void k_map_ids(const int32_t *__restrict__ perm, const int32_t *__restrict__ in, int32_t *__restrict__ out,
                          int32_t k) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) out[i] = perm[in[i]];
}
}  // namespace

void launch_map_ids(const int32_t *perm, const int32_t *in, int32_t *out, int32_t k, cudaStream_t st) {
    if (k <= 0) return;
    k_map_ids<<<(k + 255) / 256, 256, 0, st>>>(perm, in, out, k);
}

}  // namespace bcgb
