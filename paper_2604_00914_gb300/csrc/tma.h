// Tensor maps for the TMA tiled copies (cp.async.bulk.tensor): the host-side
// encoding goes through the driver's cuTensorMapEncodeTiled, reached via the
// runtime's entry-point query so that the library links only the runtime.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace apf {

// 2-D map over a row-major matrix of `rows` rows of `inner` elements of
// `dtype` (row pitch `pitch_bytes`, a multiple of 16), read in boxes of
// box_inner x box_rows elements; out-of-range parts of a box read as zero.
// Returns false when the driver entry point is missing or rejects the shape.
bool encode_tmap_2d(CUtensorMap* out, CUtensorMapDataType dtype, const void* base, uint64_t inner,
                    uint64_t rows, uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_rows,
                    CUtensorMapSwizzle swizzle);
// General tiled map of `rank` dimensions (innermost first); strides in bytes
// for dimensions 1..rank-1, each a multiple of 16.
bool encode_tmap(CUtensorMap* out, CUtensorMapDataType dtype, int rank, const void* base, const cuuint64_t* dims,
                 const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle swizzle);

}  // namespace apf
