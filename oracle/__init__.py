"""CPU oracle for the state-vector path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It shares no code with the CUDA library in
``paper_2308_01999_gb300/`` and never imports it.
"""
