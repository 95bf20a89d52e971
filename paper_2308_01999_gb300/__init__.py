"""GB300 state-vector simulator core (arXiv 2308.01999, Sec. II).

``paper_2308_01999_gb300.sv``     -- ctypes binding of ``libsv.so`` (include/sv.h)
``paper_2308_01999_gb300.inputs`` -- seeded synthetic circuits, states and Pauli strings
``paper_2308_01999_gb300._build`` -- in-tree nvcc build of ``libsv.so`` for sm_103a

Nothing is imported eagerly: importing the package loads neither torch nor the
CUDA library.
"""
