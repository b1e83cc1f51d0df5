// Temporally blocked filter kernels for f32 storage (see pm_tb.cuh).
#define AFD_TB_STORE STORE_F32
#define AFD_TB_FN(name) tb_##name##_f32
#include "pm_tb_impl.cuh"
