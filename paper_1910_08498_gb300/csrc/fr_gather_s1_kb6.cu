// Gather kernel instantiations: brick shape 1 (16 x 8 columns, 8 deep), candidate box 6x6.
#define FR_SHAPE_ID 1
#define FR_BX 16
#define FR_BY 8
#define FR_ZC 8
#define FR_KB 6
#include "fr_gather_launch.inc"
