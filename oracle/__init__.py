"""CPU FP64 oracle for the FBIM hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it and never falls back to it.

It is a plain, slow and deliberately untuned restatement of the method of
Bao, Rachh, Keaveny, Greengard & Donev, "A fluctuating boundary integral
method for Brownian suspensions" (J. Comput. Phys. 2018, arXiv:1709.01480),
in float64, written so that each step can be checked against the paper by eye:

* ``alpert``      hybrid Gauss-trapezoidal rule for log-singular integrands (Sec. 3.1, Sec. 4.1)
* ``ewald``       Hasimoto split of the periodic Stokeslet (Sec. 3.2, Eqs. HasimotoFunction,
                  wave-space-kernel, real-space-kernel, expint)
* ``singlelayer`` dense single-layer matrix M = M(t) + M(a) + M(w) (Sec. 3.2, Eqs.
                  Mwave-elements, Mreal-decompose)
* ``saddle``      K, K^T, the saddle-point system and the mobility N (Sec. 3.1,
                  Eqs. discreteSaddlePoint, discreteParticleVelocity, discreteFDB)
* ``brownian``    random slip M^1/2 W by the positive split (Sec. 3.3 and 3.4,
                  Eqs. sqrtM-split, sqrtMwave, preconditioned-real-part, Gprecond-precompute)
* ``philox``      Philox4x32-10 counter-based generator (Salmon et al., SC'11)
* ``rfd``         Euler-Maruyama step with random finite differences (Sec. 4.4, Eq. EM-RFD)
* ``mlp``         pair-correction network, its loss gradient and Adam (learned coarse level)
* ``coarse``      close body pairs, their features, two-body mobility corrections and the
                  coarse-level body velocities (learned coarse level on top of Sec. 3.4)

Parity status of each function is stated in its module header.  The wave
space is evaluated as a direct non-uniform Fourier sum: no grid, no Gaussian
spreading, no FFT and no cell list appear anywhere in this package.
"""
