// Group shapes (threads per instance, columns per thread) compiled into the
// library.  Shared by the launcher translation units and the scheduler.
#pragma once

#define OT_GROUP_SHAPES(X) \
  X(0, 32, 1)              \
  X(1, 32, 2)              \
  X(2, 32, 4)              \
  X(3, 32, 8)              \
  X(4, 64, 4)              \
  X(5, 128, 2)             \
  X(6, 128, 4)             \
  X(7, 256, 2)             \
  X(8, 256, 4)             \
  X(9, 512, 2)             \
  X(10, 512, 4)            \
  X(11, 1024, 2)           \
  X(12, 1024, 4)

#define OT_NUM_GROUP_SHAPES 13
