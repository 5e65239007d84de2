"""B300-native event-parallel tree-level matrix elements (arXiv 2312.02898 hot path).

* ``binding``     -- Python binding of the C ABI in include/me.h (libme_b300.so)
* ``phasespace``  -- seeded synthetic inputs (Philox4x32-10, RAMBO)
* ``serving``     -- continuous-batching request loop over the C ABI
* ``gen``         -- build-time process generator (diagrams, colour, CUDA emission)
* ``build``       -- build step (generate + nvcc for sm_103a + link)
"""
