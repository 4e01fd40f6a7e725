"""GB300-native time stepper for the mode-decomposed (2+1)-D Teukolsky
equation (Khanna & McKennon, arXiv:0909.4039, Sec. 2).

The compute path is the C-ABI library ``libteuk.so`` (hand-written sm_103a
CUDA, declared in ``include/teuk.h``); :mod:`paper_0909_4039_gb300.teuk` is
its thin ctypes binding.  Importing this package does not load the library,
so the seeded input generators in :mod:`paper_0909_4039_gb300.inputs` can be
used without a GPU.

Modules: ``teuk`` (the binding, ``Stepper`` and ``Batch``), ``adjoint``
(waveform-loss gradients, ``waveform_fn`` for autograd), ``sharding``
(instances over ranks), ``slabs`` (one grid as r* slabs with halo rows),
``inputs`` (seeded synthetic workloads).
"""

__all__ = ["adjoint", "inputs", "sharding", "slabs", "teuk"]
