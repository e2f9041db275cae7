// Direct-drain gather instantiations: brick shape 1 (16 x 8 columns, 8 deep).
#define FR2_SHAPE_ID 1
#define FR2_BX 16
#define FR2_BY 8
#define FR2_ZC 8
#include "fr_gather2_launch.inc"
