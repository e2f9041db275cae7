// Gather kernel instantiations: brick shape 3 (16 x 16 columns, 4 deep), candidate box 4x4.
#define FR_SHAPE_ID 3
#define FR_BX 16
#define FR_BY 16
#define FR_ZC 4
#define FR_KB 4
#include "fr_gather_launch.inc"
