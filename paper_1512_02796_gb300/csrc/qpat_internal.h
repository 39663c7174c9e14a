// Internal data structures shared by the host mesh preparation, the CUDA
// kernels and the C ABI layer.  Nothing here is part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qpat.h"

namespace qpat {

// Counts kernel launches of this library (one per launch statement; a
// replayed CUDA graph counts its kernel nodes); read by qpat_launch_count.
void note_launch(int n = 1);

// Lets kernel `func` launch with `smem` bytes of dynamic shared memory.  The
// attribute this sets is one value per kernel for the whole process, so it is
// raised once to everything the device allows beside the kernel's static
// shared memory (never lowered): concurrent launches of the same kernel from
// several host threads with different sizes then cannot undo each other.
// cudaErrorInvalidValue if `smem` exceeds that limit.
cudaError_t allow_smem(const void* func, size_t smem);

// Host-side mesh after preparation.  Node ids inside are LIBRARY ids: nodes
// are sorted by the Morton code of their coordinates, so that a contiguous
// range of library ids is a spatially compact block.  The ranges of
// `patch_nodes` consecutive library nodes are the CTA patches: a patch owns
// its range, lists every tet that touches an owned node (tets on a patch
// border appear in several patches) and the halo nodes those tets reach.
struct HostMesh {
    int64_t N = 0, E = 0, F = 0;
    int P = 0;                        // number of patches
    int patch_nodes = 0;              // target owned nodes per patch (multiple of 32)
    std::vector<int32_t> patch_of_slice;  // patch owning each 32-node slice
    std::vector<double> xyz;          // N x 3, library order
    std::vector<int32_t> tets;        // E x 4, library ids
    std::vector<int32_t> perm;        // library id -> caller id
    std::vector<int32_t> iperm;       // caller id -> library id
    std::vector<int32_t> faces_caller;  // F x 3 canonical order, caller ids ascending
    std::vector<int32_t> faces_lib;     // F x 3 same faces, library ids
    std::vector<double> farea;          // F
    // patches (CSR-style offsets, P + 1 entries each)
    std::vector<int32_t> own_begin;     // owned library range [own_begin[p], own_begin[p+1])
    std::vector<int32_t> node_ptr;      // touched nodes of patch p: nodes[node_ptr[p] ..)
    std::vector<int32_t> nodes;         //   owned ones first (in order), then halo ascending
    std::vector<int32_t> tet_ptr;
    std::vector<uint16_t> tet_loc;      // 4 local vertex ids per patch tet
    std::vector<int32_t> face_ptr;
    std::vector<uint16_t> face_loc;     // 4 per patch face: 3 local ids + 0 pad
    std::vector<double> pface_area;     // per patch face
    // Colours of each patch's tets and faces: within a colour no two share an
    // owned vertex, and each patch's list is sorted by colour.  Colour c of
    // patch p spans tets [tcol_off[j], tcol_off[j + 1]) with j = tcol_beg[p] + c,
    // j + 1 < tcol_beg[p + 1] (faces likewise with fcol_*).  Element kernels
    // run the colours one after the other, so their sums into owned rows need
    // no atomics and add up in a fixed order (run-to-run identical results).
    std::vector<int32_t> tcol_beg, tcol_off, fcol_beg, fcol_off;
    int max_tcolors = 0;
    // boundary faces of each node (library order, CSR): the load vector is
    // gathered per node in a fixed order
    std::vector<int32_t> nface_ptr, nface;
    int max_touched = 0, max_own = 0, max_ptets = 0, max_pfaces = 0;
    double extent = 0.0;                // largest bounding-box side
    // Assembled-operator pattern in sliced ELLPACK form (slices of 32
    // consecutive library rows; entry k of row 32 s + lane sits at
    // (sell_ptr[s] + k) * 32 + lane).  Column ids are LOCAL ids of the row's
    // patch (the patch's touched-node numbering), padding entries repeat the
    // row's own local id with a zero value.
    int64_t nslices = 0;
    std::vector<int64_t> sell_ptr;      // nslices + 1, in units of 32 entries
    std::vector<uint16_t> sell_col;     // 32 * sell_ptr[nslices]
    std::vector<uint8_t> sell_len;      // row lengths (32 * nslices; 0 past row N - 1)
    std::vector<int32_t> sell_diag;     // k of the diagonal entry of each row (N)
    int sell_wmax = 0;                  // widest slice (entries per row)
    // The same layout for the pure stiffness operators of the prior
    // (M(u), Eq. (14)): only pairs whose gradient coupling grad(lambda_a) .
    // grad(lambda_b) is non-zero in some tet they share.  On Kuhn meshes the
    // face- and body-diagonal edges couple with exactly zero (7 of the 15
    // entries per row remain); on general meshes the pattern equals the full one.
    std::vector<int64_t> psell_ptr;
    std::vector<uint16_t> psell_col;
    std::vector<uint8_t> psell_len;
    std::vector<int32_t> psell_diag;
    int psell_wmax = 0;
};

// Builds a HostMesh; returns "" on success or an error message.
std::string build_host_mesh(const double* xyz, int64_t N, const int32_t* tets,
                            int64_t E, int patch_nodes, int patch_multiple, HostMesh& out);

// Flux of a square boundary patch in canonical face order (see qpat.h).
void flux_patch_host(const HostMesh& m, const double c[3], const double n[3],
                     double half_w, double amp, double* flux_face);
// Flux through the curved side of a cylinder in canonical face order (see qpat.h).
void flux_side_host(const HostMesh& m, const double c[3], const double axis[3], const double ref[3],
                    double radius, double theta0, double half_w, double amp, double* flux_face);

// Plain-old-data view of the device copy of a mesh, passed to kernels by value.
struct MeshDev {
    int N, E, F, P;
    int max_touched, max_own, max_ptets, max_pfaces;
    const double* xyz64;        // N x 3 library order
    const float* xyz32;
    const int* own_begin;       // P + 1
    const int* node_ptr;        // P + 1
    const int* nodes;
    const int* tet_ptr;         // P + 1
    const ushort4* tet_loc;
    const int* face_ptr;        // P + 1
    const ushort4* face_loc;
    const int* tcol_beg;        // P + 1 (see HostMesh)
    const int* tcol_off;
    const int* fcol_beg;        // P + 1
    const int* fcol_off;
    const int* nface_ptr;       // N + 1: boundary faces of each node
    const int* nface;
    const double* pface_area64;
    const float* pface_area32;
    const int* faces_lib;       // F x 3 canonical order
    const double* farea;        // F
    const int* perm;            // library -> caller
    const int* iperm;           // caller -> library
    // sliced-ELLPACK pattern of the assembled operators (see HostMesh)
    const int64_t* sell_ptr;
    const uint16_t* sell_col;
    const uint8_t* sell_len;
    const int* sell_diag;
    int64_t sell_entries;       // 32 * sell_ptr[nslices]
    int sell_wmax;              // widest slice
};

}  // namespace qpat
