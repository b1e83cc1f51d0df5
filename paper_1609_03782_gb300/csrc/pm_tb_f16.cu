// Temporally blocked filter kernels for f16 storage (see pm_tb.cuh).
#define AFD_TB_STORE STORE_F16
#define AFD_TB_FN(name) tb_##name##_f16
#include "pm_tb_impl.cuh"
