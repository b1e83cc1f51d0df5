// Temporally blocked filter kernels for i16 storage (see pm_tb.cuh).
#define AFD_TB_STORE STORE_I16
#define AFD_TB_FN(name) tb_##name##_i16
#include "pm_tb_impl.cuh"
