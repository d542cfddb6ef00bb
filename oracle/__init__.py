"""FP64 CPU oracle for the coherent-dedispersion path -- TEST INFRASTRUCTURE ONLY.

Imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``; never by the engine.  See ``oracle.pcd`` for the path.
"""
