// ews_stencil_t4.cu -- the plain forward passes of ews_stencil.cu with
// 32 x 4 tiles (one of the tile shapes the run-time tuner chooses from).
#define EWS_TILE_Y 4
#define EWS_ROWS 1
#define EWS_SHAPE_NS t32x4
#include "ews_stencil.cu"
