// ews_stencil_t16.cu -- the plain forward passes of ews_stencil.cu with
// 32 x 16 tiles, two vertically adjacent cells per thread (one of the tile
// shapes the run-time tuner chooses from).
#define EWS_TILE_Y 16
#define EWS_ROWS 2
#define EWS_SHAPE_NS t32x16
#include "ews_stencil.cu"
