"""FP64 CPU oracle for the modulated-pyramid single-conjugate AO loop.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
execute anything in this package. The product (the CUDA library and its Python
binding in ``paper_1607_07624_gb300``) never imports it and shares no code with it.

The PASSATA paper (Agapito, Puglisi, Esposito, SPIE 2016) names the processing
objects of its loop (Table 1 parameter file, Table 2 main file: atmosphere,
propagation, modulated pyramid, CCD, slope computer, modal reconstructor,
integrator control, DM) and its GPU areas (Sec. "GPU acceleration"), but prints no
formula. The functions here are the textbook Fourier-optics and control definitions
of those objects, written plainly and slowly in FP64:

  optics      pupil stop, centred unitary DFT, four-face pyramid mask, modulation,
              detector binning, valid sub-apertures, normalised slopes
  atmosphere  von Karman phase screens by the FFT method, wind shift (bilinear)
  modal       Zernike modal basis, push-pull interaction matrix, pseudo-inverse
  control     integrator, residual wavefront error, closed loop
  noise       Philox-4x32-10 counter RNG, Poisson and Gaussian detector noise

Readings where the paper is silent are stated in each docstring. Parity status:
every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force or published known-answer vectors; the absolute fidelity
of the model to the PASSATA code itself is "parity unpinned" (the paper prints no
numbers for it).
"""
