// Marching-cubes case table (built on the host, copied to the device).
#pragma once

#include <cstdint>

namespace bcmc {

constexpr int kMaxTriPerCell = 5;   // the rule in mc_tables.cu never needs more (checked when built)

struct McTables {
    uint8_t num_tri[256];
    uint8_t tri_edges[256][16];      // 3 edge numbers per triangle, kMaxTriPerCell triangles
    int max_tri;
};

// Returns false if the rule produced something inconsistent (never expected).
bool build_mc_tables(McTables *t);

}  // namespace bcmc
