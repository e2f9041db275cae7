// Direct-drain gather instantiations: brick shape 2 (16 x 8 columns, 16 deep).
#define FR2_SHAPE_ID 2
#define FR2_BX 16
#define FR2_BY 8
#define FR2_ZC 16
#include "fr_gather2_launch.inc"
