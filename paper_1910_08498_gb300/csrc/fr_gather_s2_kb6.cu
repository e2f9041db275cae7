// Gather kernel instantiations: brick shape 2 (32 x 8 columns, 4 deep), candidate box 6x6.
#define FR_SHAPE_ID 2
#define FR_BX 32
#define FR_BY 8
#define FR_ZC 4
#define FR_KB 6
#include "fr_gather_launch.inc"
