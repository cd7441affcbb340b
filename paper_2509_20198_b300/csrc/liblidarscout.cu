// Single translation unit of liblidarscout.so: device globals (the sticky status
// word, fixed scratch arrays) exist exactly once without relocatable device code.
#include "ls_runtime.cu"
#include "ls_bin.cu"
#include "ls_fill.cu"
#include "ls_tune.cu"
#include "ls_interp.cu"
#include "ls_render.cu"
#include "ls_conv.cu"
#include "ls_wgrad.cu"
#include "ls_unet.cu"
#include "ls_cnn.cu"
#include "ls_learned.cu"
