/* fastgrid.c -- a fast seeded jittered-grid generator for streams of many
 * large synthetic meshes (the served workload), with the same construction
 * as meshgen.jittered_grid: an nx x ny vertex grid of spacing h, each quad
 * split along a coin-flipped diagonal (v00-v11 or v10-v01, triangles counter-
 * clockwise before jitter), interior nodes displaced by U(-J h, J h) in x and
 * y, the outer ring flagged fixed, nodes numbered along the Z-order (Morton)
 * curve of their grid indices or row by row.
 *
 * Random numbers come from a counter-based generator, the splitmix64
 * finaliser (Steele, Lea and Flood 2014) of seed + k * 0x9E3779B97F4A7C15
 * for draw k of one of three streams (x jitter, y jitter, diagonals), so
 * every mesh is a pure function of (nx, ny, J, seed) and can be made on any
 * thread.  It does not reproduce numpy's PCG64 draws of jittered_grid: the
 * meshes are of the same kind, not the same meshes.
 *
 * This file holds no smoothing arithmetic; it only makes inputs. */
#include <stdint.h>
#include <stdlib.h>

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t draw(uint64_t seed, uint64_t stream, uint64_t k)
{
    return mix64(seed + (stream << 58) + (k + 1) * 0x9E3779B97F4A7C15ull);
}

/* uniform in [0, 1) with 53 random bits */
static double unit(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

/* the bits of v spread to the even bit positions */
static uint64_t spread(uint64_t v)
{
    v &= 0xFFFFFFFFull;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

static int popcount64(uint64_t v)
{
    int c = 0;
    while (v) {
        v &= v - 1;
        ++c;
    }
    return c;
}

/* Morton ranks of the grid nodes (rank[j * nx + i]): the rank of a node is
 * the number of grid nodes with a smaller Z-order code, counted on a bitmap
 * of the codes of the enclosing power-of-two square.  Returns 0, or -1 when
 * out of memory. */
static int morton_ranks(int64_t nx, int64_t ny, int32_t *rank)
{
    int64_t side = 1;
    while (side < nx || side < ny) side <<= 1;
    const uint64_t words = ((uint64_t)side * (uint64_t)side + 63) / 64;
    uint64_t *bits = (uint64_t *)calloc(words, sizeof(uint64_t));
    int32_t *before = (int32_t *)malloc(sizeof(int32_t) * words);
    if (!bits || !before) {
        free(bits);
        free(before);
        return -1;
    }
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            const uint64_t c = spread((uint64_t)i) | (spread((uint64_t)j) << 1);
            bits[c >> 6] |= 1ull << (c & 63);
        }
    int32_t acc = 0;
    for (uint64_t w = 0; w < words; ++w) {
        before[w] = acc;
        acc += popcount64(bits[w]);
    }
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            const uint64_t c = spread((uint64_t)i) | (spread((uint64_t)j) << 1);
            const uint64_t below = bits[c >> 6] & ((1ull << (c & 63)) - 1ull);
            rank[j * nx + i] = before[c >> 6] + popcount64(below);
        }
    free(bits);
    free(before);
    return 0;
}

/* xy: 2 nx ny doubles; tri: 3 * 2 (nx-1)(ny-1) int32; boundary: nx ny bytes.
 * Returns 0, or -1 on bad arguments or out of memory. */
int fastgrid(int64_t nx, int64_t ny, double jitter, double h, uint64_t seed, int morton, double *xy,
             int32_t *tri, uint8_t *boundary)
{
    if (nx < 2 || ny < 2 || !xy || !tri || !boundary) return -1;
    const int64_t n = nx * ny;
    if (n >= ((int64_t)1 << 31)) return -1;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!rank) return -1;
    if (morton) {
        if (morton_ranks(nx, ny, rank) != 0) {
            free(rank);
            return -1;
        }
    } else {
        for (int64_t g = 0; g < n; ++g) rank[g] = (int32_t)g;
    }
    for (int64_t j = 0; j < ny; ++j) {
        for (int64_t i = 0; i < nx; ++i) {
            const int64_t g = j * nx + i;
            const int fixed = i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
            double x = (double)i * h, y = (double)j * h;
            if (!fixed && jitter > 0.0) {
                x = x + (2.0 * unit(draw(seed, 0, (uint64_t)g)) - 1.0) * (jitter * h);
                y = y + (2.0 * unit(draw(seed, 1, (uint64_t)g)) - 1.0) * (jitter * h);
            }
            const int32_t v = rank[g];
            xy[2 * (int64_t)v] = x;
            xy[2 * (int64_t)v + 1] = y;
            boundary[v] = (uint8_t)fixed;
        }
    }
    int64_t t = 0;
    for (int64_t j = 0; j + 1 < ny; ++j) {
        for (int64_t i = 0; i + 1 < nx; ++i) {
            const int64_t q = j * (nx - 1) + i;
            const int32_t v00 = rank[j * nx + i], v10 = rank[j * nx + i + 1];
            const int32_t v01 = rank[(j + 1) * nx + i], v11 = rank[(j + 1) * nx + i + 1];
            int32_t *a = tri + 6 * t;
            if (draw(seed, 2, (uint64_t)q) & 1u) { /* diagonal v10-v01 */
                a[0] = v00; a[1] = v10; a[2] = v01;
                a[3] = v10; a[4] = v11; a[5] = v01;
            } else { /* diagonal v00-v11 */
                a[0] = v00; a[1] = v10; a[2] = v11;
                a[3] = v00; a[4] = v11; a[5] = v01;
            }
            ++t;
        }
    }
    free(rank);
    return 0;
}
