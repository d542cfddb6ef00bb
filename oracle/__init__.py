"""FP64 CPU oracles -- TEST INFRASTRUCTURE ONLY.

Imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU legs of
``bench.py``; never by the engine.  ``oracle.pcd``: the phase-coherent path
(Sec. 3.7) with the adding-in-phase input; ``oracle.incoherent``: the AID / CID
modes (Sec. 3.4); ``oracle.ips``: the scintillation mode (Sec. 3.5);
``oracle.stack``: folding with a phase model into pulse stacks;
``oracle.boxcar`` and ``oracle.cnn``: the single-pulse detector and classifier.
"""
