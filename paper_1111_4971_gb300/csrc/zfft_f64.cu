// FP64 instantiation of the z-axis transforms.
#define PP_Z_TYPE double
#include "zfft.cu"
