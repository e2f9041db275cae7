// Gather kernel instantiations: brick shape 0 (16 x 16 columns, 8 deep), candidate box 4x4.
#define FR_SHAPE_ID 0
#define FR_BX 16
#define FR_BY 16
#define FR_ZC 8
#define FR_KB 4
#include "fr_gather_launch.inc"
