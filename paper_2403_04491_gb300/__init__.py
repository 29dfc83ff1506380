"""GB300-native KNP-EMI time step: a C-ABI CUDA library (libknp.so) and its Python binding.

The binding (``paper_2403_04491_gb300.knp``) only marshals arguments; every step of the
membrane update, assembly, AMG V-cycle and FGMRES runs in the library's CUDA kernels.
"""
from .knp import (  # noqa: F401
    KnpError, Mesh, Problem, load_library, problem_from_config, KNP_PREC_FP32, KNP_PREC_FP64,
)
from .autograd import KNPFunction, Simulation, probe_weights  # noqa: F401,E402
