// Direct-drain gather instantiations: brick shape 0 (16 x 16 columns, 8 deep).
#define FR2_SHAPE_ID 0
#define FR2_BX 16
#define FR2_BY 16
#define FR2_ZC 8
#include "fr_gather2_launch.inc"
