// internal.h -- shared declarations of the slsmooth library (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "slsmooth.h"

#ifdef __CUDACC__
#define SLS_HOST_DEVICE __host__ __device__
#else
#define SLS_HOST_DEVICE
#endif

namespace sls {

// Thread-local error message behind sls_last_error().
void set_error(const std::string &msg);
sls_status fail(sls_status code, const std::string &msg);

// Per-node adjacency word layout (one uint32 stream per mesh):
//   adj[node_off[i]]                 meta: bit 31 fixed, bits 16..30 number of
//                                    incident triangles, bits 0..15 degree
//   adj[node_off[i] + 1 ...]         the degree neighbour ids in summation order
//   adj[node_off[i] + 1 + deg ...]   one code per incident triangle:
//                                    bits 30..31 slot of node i in the stored
//                                    triangle, bits 15..29 and 0..14 the
//                                    positions (in the neighbour list) of the
//                                    other two vertices, in stored order
// A fixed node has only its meta word.
constexpr uint32_t META_FIXED = 0x80000000u;
constexpr int MAX_DEGREE = 32767;

inline uint32_t meta_word(bool fixed, uint32_t deg, uint32_t ntri)
{
    return (fixed ? META_FIXED : 0u) | (ntri << 16) | deg;
}
inline uint32_t tri_code(uint32_t slot, uint32_t pa, uint32_t pb)
{
    return (slot << 30) | (pa << 15) | pb;
}

struct HostMesh {
    int64_t n = 0, m = 0, n_free = 0;
    double diag = 0.0;                 // bounding-box diagonal of the input coordinates
    std::vector<uint32_t> node_off;    // n + 1
    std::vector<uint32_t> adj;         // node_off[n] words
    std::vector<uint8_t> fixed;        // n
};

// Processing order of the free nodes of one Form-B colour class: the class's
// nodes in ascending id, built tile by tile (kOrderTile consecutive ids per
// block).  Id order keeps a warp's reads and in-place writes close together;
// sorting by degree inside a tile was slower (scattered accesses).
constexpr int kOrderTile = 1024;

// Seed of the Form-B colouring priorities: node i has priority
// splitmix64(kColourSeed + i).
constexpr unsigned long long kColourSeed = 150200355ull;

// sqrt((xmax - xmin)^2 + (ymax - ymin)^2), the bounding-box diagonal D.
double bbox_diagonal(double xmin, double xmax, double ymin, double ymax);

// Validates the mesh and builds the adjacency stream (neighbour finding and
// constraints).  Uses up to `threads` host threads (0 = hardware concurrency).
sls_status build_host_mesh(const double *xy, int64_t n, const int32_t *tri, int64_t m,
                           const uint8_t *boundary, HostMesh &out, int threads = 0);

}  // namespace sls
