// dsr_check.cuh -- descriptor checks shared by the host entry points and
// the kernels that read descriptors from device memory (batched and served
// launches check every descriptor before running it, so a malformed one
// turns into DSR_ERR_INVALID in its teams' statuses instead of a fault).
#pragma once

#include <cstdint>

#include "dsr.h"

#ifdef __CUDACC__
#define DSR_HD __host__ __device__ __forceinline__
#else
#define DSR_HD inline
#endif

namespace dsr {

DSR_HD uint64_t pad16(uint64_t n) { return (n + 15u) & ~static_cast<uint64_t>(15u); }

DSR_HD uint32_t desc_width(const dsr_region_desc &d) {
  const uint32_t w = d.threads > 32u ? d.threads - 32u : 1u;
  return d.width ? d.width : w;
}

// 0 when the descriptor is well formed; otherwise a short reason code
// (1 shape, 2 frame sizes, 3 alignment, 4 program layout, 5 unknown program).
DSR_HD int shape_error(const dsr_region_desc &d) {
  if (d.teams == 0 || d.teams > 0x7fffffffu) return 1;
  if (d.threads < 32 || d.threads > DSR_MAX_THREADS || d.threads % 32) return 1;
  if (d.depth == 0 || d.depth > DSR_MAX_DEPTH) return 1;
  const uint32_t wmax = d.threads > 32u ? d.threads - 32u : 1u;
  if (d.width > wmax) return 1;
  for (uint32_t k = 0; k < d.depth; ++k)
    if (d.frame_bytes[k] == 0 || d.frame_bytes[k] % 4 || d.frame_bytes[k] > 0x40000000u) return 2;
  if (d.image_offset % 16 || d.out_offset % 16) return 3;
  const uint32_t w = desc_width(d);
  switch (d.program) {
    case DSR_PROG_PAPER_SCALARS:
      if (d.depth != 1 || d.param == 0 || d.param > 4096 ||
          d.frame_bytes[0] != ((4u * d.param + 7u) & ~7u) + 8u)
        return 4;
      return 0;
    case DSR_PROG_PAPER_ARRAYS:
      if (d.depth != 1 || d.param == 0 || d.param > 4096 || d.frame_bytes[0] != 4u * d.param * w)
        return 4;
      return 0;
    case DSR_PROG_SCALARS:
      return (d.depth != 1 || d.frame_bytes[0] != 16 || d.param == 0) ? 4 : 0;
    case DSR_PROG_NESTED:
      for (uint32_t k = 0; k < d.depth; ++k)
        if (d.frame_bytes[k] != 1088) return 4;
      return (d.param == 0 || static_cast<uint64_t>(d.teams) * d.param > 0xffffffffull) ? 4 : 0;
    case DSR_PROG_SWEEP:
      return d.depth != 1 ? 4 : 0;
    case DSR_PROG_HETERO:
      return 0;
    case DSR_PROG_WORKERS:
      return (d.depth != 2 || d.frame_bytes[0] != 16 || d.threads < 64 || d.param > 1) ? 4 : 0;
    default:  // a user-written program (dsr_device.cuh) states its own layout
      return d.program >= DSR_PROG_USER ? 0 : 5;
  }
}

// Input-image bytes, output bytes and status entries of a well-formed
// descriptor of a built-in program (a user-written program's images and
// outputs are its own: both 0 here).
DSR_HD void extent(const dsr_region_desc &d, uint64_t *ib, uint64_t *ob, uint64_t *ns) {
  const uint64_t T = d.teams, w = desc_width(d);
  uint64_t i = 0, o = 0;
  switch (d.program) {
    case DSR_PROG_PAPER_SCALARS:
    case DSR_PROG_PAPER_ARRAYS: o = 4 * T * w; break;
    case DSR_PROG_SCALARS: i = 16ull * d.param; o = 4ull * d.param * T * w; break;
    case DSR_PROG_NESTED: i = T * d.depth * 1088ull; o = 4 * T * d.param; break;
    case DSR_PROG_SWEEP: i = T * d.frame_bytes[0]; o = 4 * T * w; break;
    case DSR_PROG_HETERO:
      for (uint32_t k = 0; k < d.depth; ++k) i += pad16(d.frame_bytes[k]);
      o = 4 * T * w;
      break;
    case DSR_PROG_WORKERS: i = T * (16u + pad16(d.frame_bytes[1])); o = 4 * T * w; break;
  }
  *ib = i;
  *ob = o;
  *ns = T;
}

// Peak stack bytes of a well-formed descriptor's teams, and the slab that
// holds all of them under the placement rules (first fit; the worker
// program's warp stacks get even shares of the slab left after the master's
// 16-byte frame).
DSR_HD void footprint(const dsr_region_desc &d, uint64_t *stack, uint64_t *slab) {
  uint64_t st = 0, sl = 0;
  switch (d.program) {
    case DSR_PROG_WORKERS: {
      const uint64_t W = d.threads - 32u, w = desc_width(d), fp = pad16(d.frame_bytes[1]);
      const uint64_t per_warp = w < 32u ? w : 32u;
      st = 16u + w * fp;
      sl = 16u + (W / 32u) * per_warp * fp;
      break;
    }
    default:  // every frame live at the deepest point
      for (uint32_t k = 0; k < d.depth; ++k) st += pad16(d.frame_bytes[k]);
      sl = st;
  }
  *stack = st;
  *slab = sl;
}

// Bytes per team that a slab of `slab` bytes leaves to the overflow slab
// (which is assumed large enough): first fit in push order; for the worker
// program, the master's frame first and then each warp's frames in its
// even share of what is left.
DSR_HD uint64_t spill_bytes(const dsr_region_desc &d, uint64_t slab) {
  uint64_t sp = 0, spill = 0;
  if (d.program == DSR_PROG_WORKERS) {
    if (slab >= 16u) sp = 16u; else spill = 16u;
    const uint64_t W = d.threads - 32u, w = desc_width(d), fp = pad16(d.frame_bytes[1]);
    const uint64_t nwarps = W / 32u, share = ((slab - sp) / nwarps) & ~static_cast<uint64_t>(15u);
    for (uint64_t t0 = 0; t0 < w; t0 += 32u) {
      const uint64_t lanes = w - t0 < 32u ? w - t0 : 32u, fit = share / fp;
      spill += (lanes > fit ? lanes - fit : 0u) * fp;
    }
    return spill;
  }
  for (uint32_t k = 0; k < d.depth; ++k) {
    const uint64_t fp = pad16(d.frame_bytes[k]);
    if (sp + fp <= slab) sp += fp; else spill += fp;
  }
  return spill;
}

// The descriptor fits the buffers it indexes.
DSR_HD bool fits(const dsr_region_desc &d, uint64_t image_bytes, uint64_t out_bytes,
                 uint64_t n_status) {
  uint64_t ib, ob, ns;
  extent(d, &ib, &ob, &ns);
  if (ib && (d.image_offset > image_bytes || ib > image_bytes - d.image_offset)) return false;
  if (d.out_offset > out_bytes || ob > out_bytes - d.out_offset) return false;
  return static_cast<uint64_t>(d.status_index) + ns <= n_status;
}

}  // namespace dsr
