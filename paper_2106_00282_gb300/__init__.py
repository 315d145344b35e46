"""GB300 (sm_103a) split time step of the reduced two-temperature
Baer-Nunziato model (arXiv:2106.00282): CUDA kernels behind the C ABI of
include/dim.h, a ctypes binding (``api.Solver``) and seeded input generators
(``inputs``)."""
