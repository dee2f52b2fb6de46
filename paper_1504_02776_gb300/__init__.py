"""GB300-native neutron ray tracing (the hot path of MCViNE, Lin et al.).

`binding` mirrors the C ABI of libmcv.so (include/mcv.h) and fails to import when the
library is not built (there is no CPU fallback); `api` builds its structures from workload
descriptions and manages torch device buffers; `build` compiles the library.
"""
