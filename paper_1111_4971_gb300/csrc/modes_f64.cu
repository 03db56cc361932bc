// FP64 instantiation of the mode-space solve.
#define PP_M_TYPE double
#include "modes.cu"
