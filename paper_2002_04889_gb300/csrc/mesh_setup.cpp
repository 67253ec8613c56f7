// Host preparation of an uploaded mesh: orientation, local face order, face
// adjacency, FP64 cell geometry, locality renumbering (Morton / Hilbert / reverse
// Cuthill-McKee), and the partition of renumbered cells into thread-block
// sized groups with their halos.
//
// Compiled with -ffp-contract=off: the geometry below is evaluated exactly in
// the order written, so FP64 runs of the device kernels see the same bits as
// any other program that evaluates the same formulas in the same order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "../../include/volna_gb.h"
#include "vg_internal.h"

namespace vg {

namespace {

// LSD radix sort of (key, value) by 64-bit key, 8 bits per pass over the
// significant bits only; stable, so equal keys keep their value order.
void radix_sort_pairs(std::vector<uint64_t> &key, std::vector<int32_t> &val, int key_bits)
{
    size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<int32_t> v2(n);
    for (int shift = 0; shift < key_bits; shift += 8) {
        size_t count[257] = {0};
        for (size_t i = 0; i < n; i++) count[((key[i] >> shift) & 255u) + 1]++;
        for (int b = 0; b < 256; b++) count[b + 1] += count[b];
        for (size_t i = 0; i < n; i++) {
            size_t d = count[(key[i] >> shift) & 255u]++;
            k2[d] = key[i];
            v2[d] = val[i];
        }
        key.swap(k2);
        val.swap(v2);
    }
}

// Spread the low 21 bits of x to the even bit positions (bit i -> bit 2i).
uint64_t spread_bits21(uint64_t x)
{
    x &= 0x1FFFFFull;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// Z-order of cell centroids; ties keep the original order.
void morton_order(const std::vector<double> &cx, const std::vector<double> &cy,
                  std::vector<int32_t> &old_of_new)
{
    size_t n = cx.size();
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (size_t i = 0; i < n; i++) {
        x0 = std::min(x0, cx[i]); x1 = std::max(x1, cx[i]);
        y0 = std::min(y0, cy[i]); y1 = std::max(y1, cy[i]);
    }
    double span = std::max(x1 - x0, y1 - y0);
    double scale = span > 0 ? 2097151.0 / span : 0.0;
    std::vector<uint64_t> key(n);
    old_of_new.resize(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        uint64_t ix = (uint64_t)std::floor((cx[i] - x0) * scale);
        uint64_t iy = (uint64_t)std::floor((cy[i] - y0) * scale);
        key[i] = spread_bits21(ix) | (spread_bits21(iy) << 1);
        old_of_new[i] = (int32_t)i;
    }
    radix_sort_pairs(key, old_of_new, 48);
}

// Hilbert-curve order of cell centroids on a 2^21 x 2^21 grid; ties keep the
// original order.  The index is built from the most significant level down:
// each level contributes the quadrant's position along the curve, (3 rx) ^ ry
// of 0..3 times the level's cell count, then the lower bits are turned into
// the quadrant's own frame (the lower-left and lower-right quadrants are
// transposed, the latter also mirrored), so that consecutive indices are
// always neighbouring grid cells.  Blocks of consecutive cells are then
// compact, with shorter boundaries (smaller halos) than Z-order blocks.
void hilbert_order(const std::vector<double> &cx, const std::vector<double> &cy,
                   std::vector<int32_t> &old_of_new)
{
    size_t n = cx.size();
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (size_t i = 0; i < n; i++) {
        x0 = std::min(x0, cx[i]); x1 = std::max(x1, cx[i]);
        y0 = std::min(y0, cy[i]); y1 = std::max(y1, cy[i]);
    }
    double span = std::max(x1 - x0, y1 - y0);
    double scale = span > 0 ? 2097151.0 / span : 0.0;
    std::vector<uint64_t> key(n);
    old_of_new.resize(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        uint64_t x = (uint64_t)std::floor((cx[i] - x0) * scale);
        uint64_t y = (uint64_t)std::floor((cy[i] - y0) * scale);
        uint64_t d = 0;
        for (uint64_t s = 1ull << 20; s > 0; s >>= 1) {
            const uint64_t rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
            d += s * s * ((3 * rx) ^ ry);
            if (ry == 0) {
                if (rx == 1) { x = s - 1 - (x & (s - 1)); y = s - 1 - (y & (s - 1)); }
                std::swap(x, y);
            }
            x &= s - 1;
            y &= s - 1;
        }
        key[i] = d;
        old_of_new[i] = (int32_t)i;
    }
    radix_sort_pairs(key, old_of_new, 48);
}

// Reverse Cuthill-McKee on the face-adjacency graph, component by component;
// each component starts from a pseudo-peripheral cell (two BFS sweeps).
void rcm_order(const std::vector<int32_t> &nbr3, int64_t nc, std::vector<int32_t> &old_of_new)
{
    auto degree = [&](int32_t c) {
        int d = 0;
        for (int f = 0; f < 3; f++) d += nbr3[3 * (int64_t)c + f] >= 0;
        return d;
    };
    std::vector<int32_t> level(nc, -1), queue;
    std::vector<char> placed(nc, 0);
    queue.reserve(nc);
    old_of_new.clear();
    old_of_new.reserve(nc);
    std::vector<int32_t> comp;
    auto bfs_last = [&](int32_t s) {
        // BFS over the component of s; returns a min-degree cell of the last level.
        comp.clear();
        comp.push_back(s);
        level[s] = 0;
        size_t h = 0;
        while (h < comp.size()) {
            int32_t c = comp[h++];
            for (int f = 0; f < 3; f++) {
                int32_t j = nbr3[3 * (int64_t)c + f];
                if (j >= 0 && level[j] < 0) { level[j] = level[c] + 1; comp.push_back(j); }
            }
        }
        int32_t last_level = level[comp.back()];
        int32_t best = comp.back();
        for (size_t i = comp.size(); i-- > 0 && level[comp[i]] == last_level;) {
            int32_t c = comp[i];
            if (degree(c) < degree(best) || (degree(c) == degree(best) && c < best)) best = c;
        }
        for (int32_t c : comp) level[c] = -1;
        return best;
    };
    for (int64_t s0 = 0; s0 < nc; s0++) {
        if (placed[s0]) continue;
        int32_t s = bfs_last(bfs_last((int32_t)s0));
        size_t first = old_of_new.size();
        old_of_new.push_back(s);
        placed[s] = 1;
        for (size_t h = first; h < old_of_new.size(); h++) {
            int32_t c = old_of_new[h];
            int32_t nb[3];
            int k = 0;
            for (int f = 0; f < 3; f++) {
                int32_t j = nbr3[3 * (int64_t)c + f];
                if (j >= 0 && !placed[j]) nb[k++] = j;
            }
            std::sort(nb, nb + k, [&](int32_t a, int32_t b) {
                int da = degree(a), db = degree(b);
                return da != db ? da < db : a < b;
            });
            for (int i = 0; i < k; i++) { placed[nb[i]] = 1; old_of_new.push_back(nb[i]); }
        }
    }
    std::reverse(old_of_new.begin(), old_of_new.end());
}

}  // namespace

int bed_arrays(HostMesh &m, const double *depth_v, std::string &err)
{
    const int64_t nc = m.nc;
    std::vector<double> z(nc), zf(3 * (size_t)nc);
    int64_t bad = -1;
    for (int64_t k = 0; k < nc; k++) {
        const int32_t *v = &m.vtx[3 * (size_t)m.old_of_new[k]];
        z[k] = -((depth_v[v[0]] + depth_v[v[1]]) + depth_v[v[2]]) / 3.0;
        bool ok = std::isfinite(z[k]);
        for (int f = 0; f < 3; f++) {
            zf[f * (size_t)nc + k] = -(depth_v[v[f]] + depth_v[v[(f + 1) % 3]]) / 2.0;
            ok = ok && std::isfinite(zf[f * (size_t)nc + k]);
        }
        if (!ok && bad < 0) bad = m.old_of_new[k];
    }
    if (bad >= 0) { err = "triangle " + std::to_string(bad) + " has a non-finite depth"; return VG_EINVAL; }
    m.z.swap(z);
    m.zf.swap(zf);
    return VG_OK;
}

int prepare_mesh(int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                 const double *depth_v, int renumber, int block, HostMesh &m, std::string &err)
{
    if (nv < 3 || nc < 1 || !xy || !tri || !depth_v) { err = "empty mesh or NULL array"; return VG_EINVAL; }
    if (nc > (int64_t)INT32_MAX / GEO_ROWS || nv > (int64_t)INT32_MAX) {
        err = "mesh too large: at most " + std::to_string((int64_t)INT32_MAX / GEO_ROWS) + " cells";
        return VG_EINVAL;
    }
    if (renumber < 0 || renumber > 3) { err = "renumber must be 0, 1, 2 or 3"; return VG_EINVAL; }
    m = HostMesh();
    m.nc = nc;
    m.nv = nv;
    m.xy.assign(xy, xy + 2 * nv);
    m.vtx.resize(3 * nc);

    // 1. orientation (counter-clockwise) and local order (smallest vertex id first)
    int64_t flipped = 0, bad_id = -1, bad_area = -1;
#pragma omp parallel for schedule(static) reduction(+ : flipped)
    for (int64_t c = 0; c < nc; c++) {
        int32_t a = tri[3 * c], b = tri[3 * c + 1], d = tri[3 * c + 2];
        if (a < 0 || b < 0 || d < 0 || a >= nv || b >= nv || d >= nv || a == b || b == d || a == d) {
#pragma omp critical
            bad_id = bad_id < 0 ? c : std::min(bad_id, c);
            continue;
        }
        double s = (xy[2 * b] - xy[2 * a]) * (xy[2 * d + 1] - xy[2 * a + 1])
                 - (xy[2 * b + 1] - xy[2 * a + 1]) * (xy[2 * d] - xy[2 * a]);
        if (s == 0.0 || !std::isfinite(s)) {
#pragma omp critical
            bad_area = bad_area < 0 ? c : std::min(bad_area, c);
            continue;
        }
        int32_t v[3] = {a, b, d};
        if (s < 0.0) { std::swap(v[1], v[2]); flipped++; }
        int k0 = (v[1] < v[0]) ? 1 : 0;
        if (v[2] < v[k0]) k0 = 2;
        for (int k = 0; k < 3; k++) m.vtx[3 * c + k] = v[(k0 + k) % 3];
    }
    if (bad_id >= 0) { err = "triangle " + std::to_string(bad_id) + " has an out-of-range or repeated vertex id"; return VG_EINVAL; }
    if (bad_area >= 0) { err = "triangle " + std::to_string(bad_area) + " has zero area"; return VG_EINVAL; }
    m.n_flipped = flipped;

    // 2. face adjacency: match each directed edge p->q with a q->p edge.
    //    Directed edges are grouped by their start vertex (CSR).
    std::vector<int64_t> start(nv + 1, 0);
    for (int64_t i = 0; i < 3 * nc; i++) start[m.vtx[i] + 1]++;
    for (int64_t v = 0; v < nv; v++) start[v + 1] += start[v];
    std::vector<int64_t> edge_of(3 * nc);   // directed edge id = 3 c + f, grouped by start
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < 3 * nc; i++) edge_of[fill[m.vtx[i]]++] = i;
    }
    std::vector<int32_t> nbr_o(3 * nc), nface_o(3 * nc);
    int64_t bad_edge = -1;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; c++) {
        for (int f = 0; f < 3; f++) {
            int32_t p = m.vtx[3 * c + f], q = m.vtx[3 * c + (f + 1) % 3];
            int32_t found = -1, fface = -1, count = 0;
            for (int64_t k = start[q]; k < start[q + 1]; k++) {
                int64_t e = edge_of[k];
                int32_t d = (int32_t)(e / 3), g = (int32_t)(e % 3);
                if (m.vtx[3 * (int64_t)d + (g + 1) % 3] == p) { found = d; fface = g; count++; }
            }
            int same_dir = 0;
            for (int64_t k = start[p]; k < start[p + 1]; k++) {
                int64_t e = edge_of[k];
                if (e != 3 * c + f && m.vtx[3 * (e / 3) + (e % 3 + 1) % 3] == q) same_dir = 1;
            }
            if (count > 1 || same_dir || found == c) {
#pragma omp critical
                bad_edge = bad_edge < 0 ? c : std::min(bad_edge, c);
            }
            nbr_o[3 * c + f] = found;
            nface_o[3 * c + f] = fface;
        }
    }
    if (bad_edge >= 0) { err = "triangle " + std::to_string(bad_edge) + " has a non-manifold edge"; return VG_EINVAL; }

    // 3. FP64 geometry in the original order
    std::vector<double> area(nc), cx(nc), cy(nc), zc(nc);
    std::vector<double> gnx(3 * nc), gny(3 * nc), glen(3 * nc), gfx(3 * nc), gfy(3 * nc), gwx(3 * nc), gwy(3 * nc);
    int64_t bad_geo = -1;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; c++) {
        const int32_t *v = &m.vtx[3 * c];
        double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1];
        double bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
        double qx = xy[2 * v[2]], qy = xy[2 * v[2] + 1];
        area[c] = 0.5 * ((bx - ax) * (qy - ay) - (by - ay) * (qx - ax));
        cx[c] = ((ax + bx) + qx) / 3.0;
        cy[c] = ((ay + by) + qy) / 3.0;
        zc[c] = -((depth_v[v[0]] + depth_v[v[1]]) + depth_v[v[2]]) / 3.0;
        if (!(area[c] > 0.0) || !std::isfinite(zc[c])) {
#pragma omp critical
            bad_geo = bad_geo < 0 ? c : std::min(bad_geo, c);
        }
        for (int f = 0; f < 3; f++) {
            int32_t p = v[f], q = v[(f + 1) % 3];
            double ex = xy[2 * q] - xy[2 * p], ey = xy[2 * q + 1] - xy[2 * p + 1];
            double l = std::sqrt(ex * ex + ey * ey);
            glen[3 * c + f] = l;
            gnx[3 * c + f] = ey / l;
            gny[3 * c + f] = -ex / l;
            gfx[3 * c + f] = 0.5 * (xy[2 * p] + xy[2 * q]) - cx[c];
            gfy[3 * c + f] = 0.5 * (xy[2 * p + 1] + xy[2 * q + 1]) - cy[c];
        }
    }
    if (bad_geo >= 0) { err = "triangle " + std::to_string(bad_geo) + " has a degenerate area or non-finite depth"; return VG_EINVAL; }
    // least-squares weights over the three stencil offsets (neighbour centroid,
    // or the centroid reflected across a wall face)
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; c++) {
        double dx[3], dy[3];
        double Mxx = 0.0, Mxy = 0.0, Myy = 0.0;
        for (int f = 0; f < 3; f++) {
            int64_t i = 3 * c + f;
            int32_t j = nbr_o[i];
            if (j >= 0) {
                dx[f] = cx[j] - cx[c];
                dy[f] = cy[j] - cy[c];
            } else {
                double dn = gfx[i] * gnx[i] + gfy[i] * gny[i];
                dx[f] = 2.0 * dn * gnx[i];
                dy[f] = 2.0 * dn * gny[i];
            }
            Mxx = Mxx + dx[f] * dx[f];
            Mxy = Mxy + dx[f] * dy[f];
            Myy = Myy + dy[f] * dy[f];
        }
        double det = Mxx * Myy - Mxy * Mxy;
        for (int f = 0; f < 3; f++) {
            gwx[3 * c + f] = (Myy * dx[f] - Mxy * dy[f]) / det;
            gwy[3 * c + f] = (Mxx * dy[f] - Mxy * dx[f]) / det;
        }
    }

    // 4. renumbering
    if (renumber == VG_RENUMBER_MORTON) {
        morton_order(cx, cy, m.old_of_new);
    } else if (renumber == VG_RENUMBER_HILBERT) {
        hilbert_order(cx, cy, m.old_of_new);
    } else if (renumber == VG_RENUMBER_RCM) {
        rcm_order(nbr_o, nc, m.old_of_new);
    } else {
        m.old_of_new.resize(nc);
        std::iota(m.old_of_new.begin(), m.old_of_new.end(), 0);
    }
    m.new_of_old.assign(nc, -1);
    for (int64_t k = 0; k < nc; k++) m.new_of_old[m.old_of_new[k]] = (int32_t)k;

    // 5. internal-order arrays
    m.geo.resize((size_t)GEO_ROWS * nc);
    m.nbr.resize(3 * nc);
    std::vector<int32_t> nface(3 * nc);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; k++) {
        int64_t o = m.old_of_new[k];
        for (int f = 0; f < 3; f++) {
            int64_t i = 3 * o + f;
            m.geo[(GEO_NX + f) * nc + k] = gnx[i];
            m.geo[(GEO_NY + f) * nc + k] = gny[i];
            m.geo[(GEO_LEN + f) * nc + k] = glen[i];
            m.geo[(GEO_FX + f) * nc + k] = gfx[i];
            m.geo[(GEO_FY + f) * nc + k] = gfy[i];
            m.geo[(GEO_WX + f) * nc + k] = gwx[i];
            m.geo[(GEO_WY + f) * nc + k] = gwy[i];
            m.nbr[f * nc + k] = nbr_o[i] >= 0 ? m.new_of_old[nbr_o[i]] : -1;
            nface[f * nc + k] = nface_o[i];
        }
        m.geo[GEO_AREA * nc + k] = area[o];
    }
    {
        int rc = bed_arrays(m, depth_v, err);
        if (rc) return rc;
    }
    // keep the neighbour faces for partition_blocks
    m.nbrl.assign(3 * nc, NBR_WALL);
    for (int64_t i = 0; i < 3 * nc; i++) m.nbrl[i] = nface[i] >= 0 ? (uint16_t)nface[i] : NBR_WALL;
    return partition_blocks(m, block, err);
}

// Blocks of `block` consecutive cells.  Each block's halo has two rings:
// ring 1 = face neighbours of block cells outside the block (their face values
// are reconstructed by the block), ring 2 = face neighbours of ring-1 cells
// outside block and ring 1 (their states feed ring-1 gradients).  Local indices:
// block cells [0, block), ring 1 [block, block + n1), ring 2 after that.
int partition_blocks(HostMesh &m, int block, std::string &err)
{
    if (block < 32 || block > 1024 || block % 32) { err = "block_cells must be a multiple of 32 in [32, 1024]"; return VG_EINVAL; }
    int64_t nc = m.nc;
    // recover the neighbour face of each (cell, face): low 2 bits of nbrl
    std::vector<uint8_t> nface(3 * nc);
    for (int64_t i = 0; i < 3 * nc; i++) nface[i] = m.nbr[i] < 0 ? 3 : (uint8_t)(m.nbrl[i] & 3u);
    int32_t nb = (int32_t)((nc + block - 1) / block);
    m.block = block;
    m.nblocks = nb;
    std::vector<std::vector<int32_t>> r1(nb), r2(nb);
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t b = 0; b < nb; b++) {
        int64_t c0 = (int64_t)b * block, c1 = std::min<int64_t>(c0 + block, nc);
        std::vector<int32_t> &h = r1[b];
        for (int f = 0; f < 3; f++)
            for (int64_t c = c0; c < c1; c++) {
                int32_t j = m.nbr[f * nc + c];
                if (j >= 0 && (j < c0 || j >= c1)) h.push_back(j);
            }
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
        std::vector<int32_t> &h2 = r2[b];
        for (int32_t r : h)
            for (int f = 0; f < 3; f++) {
                int32_t j = m.nbr[f * nc + r];
                if (j >= 0 && (j < c0 || j >= c1) && !std::binary_search(h.begin(), h.end(), j)) h2.push_back(j);
            }
        std::sort(h2.begin(), h2.end());
        h2.erase(std::unique(h2.begin(), h2.end()), h2.end());
    }
    m.halo_ptr.assign(nb + 1, 0);
    m.halo_n1.assign(nb, 0);
    int32_t mh = 0, m1 = 0;
    for (int32_t b = 0; b < nb; b++) {
        int32_t n = (int32_t)(r1[b].size() + r2[b].size());
        m.halo_ptr[b + 1] = m.halo_ptr[b] + n;
        m.halo_n1[b] = (int32_t)r1[b].size();
        mh = std::max(mh, n);
        m1 = std::max(m1, m.halo_n1[b]);
    }
    if (block + mh >= (1 << 14) - 1) { err = "a block's halo is too large"; return VG_EINVAL; }
    m.max_halo = mh;
    m.max_ring1 = m1;
    m.halo_ids.resize(m.halo_ptr[nb]);
    m.ring1_nbr.assign(3 * (size_t)m.halo_ptr[nb], NBR_WALL);
    std::vector<uint16_t> nbrl(3 * nc, NBR_WALL);
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t b = 0; b < nb; b++) {
        int64_t c0 = (int64_t)b * block, c1 = std::min<int64_t>(c0 + block, nc);
        const std::vector<int32_t> &h = r1[b], &h2 = r2[b];
        int32_t n1 = (int32_t)h.size();
        std::copy(h.begin(), h.end(), m.halo_ids.begin() + m.halo_ptr[b]);
        std::copy(h2.begin(), h2.end(), m.halo_ids.begin() + m.halo_ptr[b] + n1);
        auto local_of = [&](int32_t j) -> int32_t {
            if (j >= c0 && j < c1) return (int32_t)(j - c0);
            auto it = std::lower_bound(h.begin(), h.end(), j);
            if (it != h.end() && *it == j) return block + (int32_t)(it - h.begin());
            it = std::lower_bound(h2.begin(), h2.end(), j);
            return block + n1 + (int32_t)(it - h2.begin());
        };
        for (int f = 0; f < 3; f++)
            for (int64_t c = c0; c < c1; c++) {
                int32_t j = m.nbr[f * nc + c];
                if (j < 0) {
                    if (j == -2) nbrl[f * nc + c] = NBR_OPEN;
                    else if (j == -3) nbrl[f * nc + c] = NBR_ABSORB;
                    continue;
                }
                nbrl[f * nc + c] = (uint16_t)((local_of(j) << 2) | nface[f * nc + c]);
            }
        for (int32_t k = 0; k < n1; k++)
            for (int f = 0; f < 3; f++) {
                int32_t j = m.nbr[f * nc + h[k]];
                uint16_t &code = m.ring1_nbr[3 * ((size_t)m.halo_ptr[b] + k) + f];
                if (j >= 0) code = (uint16_t)local_of(j);
                else if (j == -2) code = NBR_OPEN;
                else if (j == -3) code = NBR_ABSORB;
            }
    }
    m.nbrl.swap(nbrl);
    // Owned faces of each block, in cell-then-face order: a face on the domain
    // boundary, a face to the halo, or a face to a block cell of higher local
    // index (so every face of the block is computed once).  Only the face's
    // kind matters, so switching a boundary face between wall and open keeps it.
    m.fq_ptr.assign(nb + 1, 0);
    auto owned = [&](int64_t c, int64_t c0, int f) {
        const uint16_t code = m.nbrl[f * nc + c];
        return code >= NBR_ABSORB || (code >> 2) >= block || (int64_t)(code >> 2) > c - c0;
    };
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t b = 0; b < nb; b++) {
        int64_t c0 = (int64_t)b * block, c1 = std::min<int64_t>(c0 + block, nc);
        int32_t n = 0;
        for (int64_t c = c0; c < c1; c++)
            for (int f = 0; f < 3; f++) n += owned(c, c0, f);
        m.fq_ptr[b + 1] = n;
    }
    for (int32_t b = 0; b < nb; b++) m.fq_ptr[b + 1] += m.fq_ptr[b];
    m.fq.resize(std::max<int32_t>(m.fq_ptr[nb], 1));
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t b = 0; b < nb; b++) {
        int64_t c0 = (int64_t)b * block, c1 = std::min<int64_t>(c0 + block, nc);
        int32_t k = m.fq_ptr[b];
        for (int64_t c = c0; c < c1; c++)
            for (int f = 0; f < 3; f++)
                if (owned(c, c0, f)) m.fq[k++] = (uint16_t)(((c - c0) << 2) | f);
    }
    return VG_OK;
}

void locate_points(const HostMesh &m, int32_t n, const double *pts, int32_t *cells)
{
    const double *xy = m.xy.data();
    for (int32_t k = 0; k < n; k++) {
        double px = pts[2 * k], py = pts[2 * k + 1];
        int64_t best = INT64_MAX;
#pragma omp parallel for schedule(static) reduction(min : best)
        for (int64_t c = 0; c < m.nc; c++) {
            bool inside = true;
            for (int f = 0; f < 3 && inside; f++) {
                int32_t a = m.vtx[3 * c + f], b = m.vtx[3 * c + (f + 1) % 3];
                double o = (xy[2 * b] - xy[2 * a]) * (py - xy[2 * a + 1])
                         - (xy[2 * b + 1] - xy[2 * a + 1]) * (px - xy[2 * a]);
                if (o < 0.0) inside = false;
            }
            if (inside && c < best) best = c;
        }
        cells[k] = best == INT64_MAX ? -1 : (int32_t)best;
    }
}

}  // namespace vg
