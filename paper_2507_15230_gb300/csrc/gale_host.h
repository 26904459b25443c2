// Host-side state of a loaded mesh (internal).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gale.h"
#include "gale_internal.h"

namespace gale {

struct HostMesh {
    int64_t nv = 0, nt = 0;
    int32_t K = 0;
    std::vector<int32_t> cid;         // input vertex -> canonical
    std::vector<int32_t> vperm;       // canonical vertex -> input
    std::vector<int32_t> cluster_of;  // canonical vertex -> cluster
    std::vector<int32_t> tperm;       // canonical tet -> input
    std::vector<int32_t> I_V, I_T;    // [K+1]
    std::vector<int32_t> rows;        // [4 nt] canonical rows, canonical order
    std::vector<int64_t> ext_off;     // [K+1]
    std::vector<int32_t> ext;         // T_ex lists, ascending per cluster
    std::vector<int64_t> halo_off;    // [K+1]
    std::vector<int32_t> halo;        // halo lists, ascending per cluster
    std::vector<ClusterStat> stats;   // [K+NP] clusters, then parts
    std::vector<int64_t> blk_off;     // [K+NP+1] word offsets
    int32_t NP = 0;                   // parts of the cut clusters
    std::vector<PartInfo> parts;      // [NP] (the b_* fields are set after the counting pass)
    std::vector<int32_t> part_first;  // [K+1] parts of cluster k: part_first[k] .. part_first[k+1]-1
    int32_t *blocks = nullptr;        // blocks_words words (pinned when possible)
    int64_t blocks_words = 0;
    bool blocks_pinned = false;
    int64_t ext_total = 0, halo_total = 0;
    double host_seconds = 0;

    bool alloc_blocks(int64_t words);
    void free_blocks();
    ~HostMesh() { free_blocks(); }
};

int host_threads(int requested);
bool prepare_host(const gale_mesh_desc &d, HostMesh &hm, std::string &err);

}  // namespace gale
