// cx_halo.cu -- halo exchange of a sub-domain (domain decomposition of one
// problem over several devices or processes).
//
// The method's collision is local and its streaming reaches only the nearest
// neighbours (Sec. 3.1: each node's update reads the populations of x - e_i;
// the adjoint of Sec. 3.2.1 those of x + e_i), so a 2-D block partition of
// the lattice needs, before every step, the populations that cross each
// block face and corner.  A sub-domain of lx x ly nodes is stored as an
// (lx + 2) x (ly + 2) grid whose outer frame holds ghost copies of the
// neighbouring blocks' boundary nodes (descriptor field halo = 1).
//
// Slots: direction d = 1..8 names the neighbour at offset e_d (the D2Q9
// velocities: E, N, W, S, NE, NW, SW, SE).  Send slot d holds this block's
// interior cells along side d (a column or row of ly or lx cells, one cell for
// a corner) for the planes the neighbour's interior nodes pull across that
// side:
//   forward populations (kind FWD): the directions i moving toward d
//     (e_i,x = +1 for E, e_i,y = +1 for N, ..., e_i = e_d for a corner),
//     for both species: 3 + 3 planes per face and 1 + 1 per corner on D2Q9
//     (1 + 1 per face and none at corners on D2Q5);
//   adjoint populations (kind ADJ): the opposite directions (the adjoint
//     pulls from x + e_i, streaming along -e_i);
//   a node field (kind SEED, the terminal adjoint seed): the field itself.
// The neighbour at e_d stores it as its receive slot opp(d) and unpacks it
// into its ghost cells on side opp(d).  Slots are laid out one after another
// in direction order, each [planes][cells] of T.
#include <algorithm>

#include "cx_device.cuh"
#include "cx_state.h"

namespace cx {

// planes of `kind` that cross side d (d = 1..8), written to mask bits (bit j: plane j of [2][Q])
template <int Q> __host__ __device__ inline unsigned halo_planes(int kind, int d) {
    using L = Lat<9>;
    if (kind == CX_HALO_SEED) return 1u;
    const int dx = L::ex(d), dy = L::ey(d);
    unsigned m = 0;
    for (int i = 1; i < Q; ++i) {
        // forward: the pulled population moves toward the side; adjoint: away from it
        const int ex = kind == CX_HALO_FWD ? L::ex(i) : -L::ex(i);
        const int ey = kind == CX_HALO_FWD ? L::ey(i) : -L::ey(i);
        const bool cross = (dx != 0 && dy != 0) ? (ex == dx && ey == dy) : (dx != 0 ? ex == dx : ey == dy);
        if (cross) m |= (1u << i) | (1u << (Q + i));
    }
    return m;
}

struct HaloGeom {
    int lx, ly, nx;              // interior size, row stride (lx + 2)
    int nplanes[9], len[9];      // per direction d = 1..8
    unsigned planes[9];
    long long off[9];            // slot offsets in values of T
    long long plane;             // plane stride of the population buffer
    long long total;             // values of all slots
};

inline HaloGeom halo_geom(int nx, int ny, int Q, long long plane, int kind) {
    HaloGeom G{};
    G.lx = nx - 2;
    G.ly = ny - 2;
    G.nx = nx;
    G.plane = plane;
    long long o = 0;
    for (int d = 1; d <= 8; ++d) {
        const unsigned m = Q == 9 ? halo_planes<9>(kind, d) : halo_planes<5>(kind, d);
        G.planes[d] = m;
        G.nplanes[d] = __builtin_popcount(m);
        G.len[d] = d <= 4 ? ((d == 1 || d == 3) ? G.ly : G.lx) : 1;
        G.off[d] = o;
        o += (long long)G.nplanes[d] * G.len[d];
    }
    G.total = o;
    return G;
}

// local (x, y) of cell t along side d: interior boundary cells (pack) or the
// ghost cells beyond them (unpack)
__host__ __device__ inline void halo_cell(const HaloGeom& G, int d, int t, bool ghost, int* x, int* y) {
    using L = Lat<9>;
    const int dx = L::ex(d), dy = L::ey(d);
    const int xe = dx > 0 ? G.lx + (ghost ? 1 : 0) : (dx < 0 ? (ghost ? 0 : 1) : 1 + t);
    const int ye = dy > 0 ? G.ly + (ghost ? 1 : 0) : (dy < 0 ? (ghost ? 0 : 1) : 1 + t);
    *x = xe;
    *y = ye;
}

// pack: one thread per (plane, cell) of slot d = blockIdx.y + 1
template <typename T>
__global__ void k_halo_pack(HaloGeom G, const T* field, T* send) {
    const int d = blockIdx.y + 1;
    const int n = G.nplanes[d] * G.len[d];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int pj = e / G.len[d], t = e - pj * G.len[d];
        int j = -1, c = -1;
        for (int b = 0; b < 32; ++b) // the pj-th set bit of the plane mask
            if ((G.planes[d] >> b) & 1u)
                if (++c == pj) {
                    j = b;
                    break;
                }
        int x, y;
        halo_cell(G, d, t, false, &x, &y);
        send[G.off[d] + e] = field[(long long)j * G.plane + (long long)y * G.nx + x];
    }
}

// unpack: receive slot d (from the neighbour at e_d) into the ghost cells on side d
template <typename T>
__global__ void k_halo_unpack(HaloGeom G, HaloGeom S, const T* recv, T* field) {
    // S describes the sender's slots: slot opp(d) of the neighbour carries the planes of direction opp(d)
    const int d = blockIdx.y + 1;
    const int so = (d <= 4) ? ((d + 1) % 4) + 1 : ((d - 5 + 2) % 4) + 5; // opp(d)
    const int n = S.nplanes[so] * G.len[d];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int pj = e / G.len[d], t = e - pj * G.len[d];
        int j = -1, c = -1;
        for (int b = 0; b < 32; ++b)
            if ((S.planes[so] >> b) & 1u)
                if (++c == pj) {
                    j = b;
                    break;
                }
        int x, y;
        halo_cell(G, d, t, true, &x, &y);
        field[(long long)j * G.plane + (long long)y * G.nx + x] = recv[G.off[d] + e];
    }
}

} // namespace cx

using namespace cx;

namespace {

bool halo_ok(const cx_problem* p, int kind) {
    return p && p->d.halo && (kind == CX_HALO_FWD || kind == CX_HALO_ADJ || kind == CX_HALO_SEED);
}

// the receive layout: slot d holds what the neighbour at e_d packed as its slot opp(d)
HaloGeom recv_geom(const HaloGeom& S) {
    HaloGeom R = S;
    long long o = 0;
    for (int d = 1; d <= 8; ++d) {
        const int so = (d <= 4) ? ((d + 1) % 4) + 1 : ((d - 5 + 2) % 4) + 5;
        R.off[d] = o;
        o += (long long)S.nplanes[so] * S.len[d];
    }
    R.total = o;
    return R;
}

} // namespace

extern "C" {

cx_status cx_halo_layout(const cx_problem* p, int kind, size_t* send_off, size_t* recv_off, size_t* bytes) {
    if (!halo_ok(p, kind)) return CX_ERR_INVALID_ARG;
    const HaloGeom S = halo_geom(p->d.nx, p->d.ny, p->lay.Q, (long long)p->lay.plane, kind);
    const HaloGeom R = recv_geom(S);
    for (int d = 1; d <= 8; ++d) {
        if (send_off) send_off[d - 1] = (size_t)S.off[d] * p->lay.esz;
        if (recv_off) recv_off[d - 1] = (size_t)R.off[d] * p->lay.esz;
    }
    if (bytes) *bytes = (size_t)S.total * p->lay.esz;
    return CX_OK;
}

cx_status cx_halo_pack(cx_problem* p, int kind, const void* field, void* send) {
    if (!halo_ok(p, kind) || !field || !send) return CX_ERR_INVALID_ARG;
    const HaloGeom G = halo_geom(p->d.nx, p->d.ny, p->lay.Q, (long long)p->lay.plane, kind);
    const int mx = std::max(G.lx, G.ly) * 6;
    const dim3 grid((unsigned)std::max(1, (mx + 255) / 256), 8);
    if (p->lay.esz == 8)
        k_halo_pack<double><<<grid, 256, 0, p->stream>>>(G, (const double*)field, (double*)send);
    else
        k_halo_pack<float><<<grid, 256, 0, p->stream>>>(G, (const float*)field, (float*)send);
    return cudaGetLastError() == cudaSuccess ? CX_OK : CX_ERR_CUDA;
}

cx_status cx_halo_unpack(cx_problem* p, int kind, const void* recv, void* field) {
    if (!halo_ok(p, kind) || !field || !recv) return CX_ERR_INVALID_ARG;
    const HaloGeom S = halo_geom(p->d.nx, p->d.ny, p->lay.Q, (long long)p->lay.plane, kind);
    const HaloGeom R = recv_geom(S);
    const int mx = std::max(S.lx, S.ly) * 6;
    const dim3 grid((unsigned)std::max(1, (mx + 255) / 256), 8);
    if (p->lay.esz == 8)
        k_halo_unpack<double><<<grid, 256, 0, p->stream>>>(R, S, (const double*)recv, (double*)field);
    else
        k_halo_unpack<float><<<grid, 256, 0, p->stream>>>(R, S, (const float*)recv, (float*)field);
    return cudaGetLastError() == cudaSuccess ? CX_OK : CX_ERR_CUDA;
}

} // extern "C"
