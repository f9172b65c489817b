// Size limits the host checks before a lattice reaches a marching kernel.
#pragma once

#include <stddef.h>

namespace qla {

// The marching kernels (single, batched) form element offsets in 32 bits:
// every live plane of the storage, planes x plane_elems elements, must be
// addressable that way.  Lattices past it step on the tile kernel (64-bit
// offsets) or are refused where no other kernel exists (double-single,
// batches).
inline bool offsets32_ok(size_t planes, size_t plane_elems) {
    return plane_elems < (size_t(1) << 31) && planes * plane_elems <= (size_t(1) << 32);
}

// Record indices are 32-bit: a site's index is either one of the shared
// slots or shared_slots + its own record number, so the slots plus every
// site of the lattice must stay below 2^32.
inline bool record_ids_ok(size_t sites, size_t shared_slots) {
    return shared_slots + sites < (size_t(1) << 32);
}

// Elements per plane of an nx x ny lattice (rows padded to 32 elements).
inline size_t padded_plane(int nx, int ny) {
    return size_t(ny) * ((size_t(nx) + 31) / 32 * 32);
}

}  // namespace qla
