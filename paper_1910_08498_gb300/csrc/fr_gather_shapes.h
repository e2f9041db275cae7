// fr_gather_shapes.h -- the brick shapes of the gather kernel family (one
// translation unit per shape, fr_gather_s<k>.cu, so they compile in parallel).
#pragma once

// id, columns in x, columns in y, voxels per column (z)
#define FR_GATHER_SHAPES(X) \
  X(0, 16, 16, 8)           \
  X(1, 16, 8, 8)            \
  X(2, 32, 8, 4)            \
  X(3, 16, 16, 4)

#define FR_NUM_GATHER_SHAPES 4
