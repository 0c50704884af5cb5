"""Oracle: a plain, slow FP64 CPU restatement of the batched acceptance-walk
nested sampler for gravitational-wave likelihoods (arXiv 2509.04336).

This package is test infrastructure.  Only the tests, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA path; the only module both sides use is the
seeded input generator ``paper_2509_04336_gb300.synth``, which holds none of the
method's arithmetic.

Modules and the passages they follow:
  philox      counter-based RNG (Salmon et al. 2011, Philox4x64-10)
  prior       unit-cube transforms of Table 1 (Sec. 3.4)
  detector    antenna patterns and arrival-time delays of the detector network (Sec. 4.1.1)
  taylorf2    3.5PN aligned-spin TaylorF2 waveform (workload waveform; PN literature)
  phenomd     IMRPhenomD-form waveform (Sec. 3.3 names IMRPhenomD; form-only coefficient table)
  likelihood  frequency-domain Gaussian likelihood (Sec. 3.3)
  walk        DE acceptance walk under L > L* (Sec. 3.1, footnote on the DE scale)
  nested      batched nested sampling, expected shrinkage and evidence (Sec. 2.2.3, Sec. 3.2, Sec. 3.2.1)
  flow        affine-coupling flow proposal and its Adam training (motivated in Sec. 5; RealNVP)
  relbin      relative-binning (heterodyned) likelihood (named in Sec. 3.3, Sec. 5; Zackay et al. 2018)

Functions without an independent pin say "parity unpinned" in their docstring.
"""
