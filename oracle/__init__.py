"""FP64 CPU oracle for the tumor reaction-diffusion calibration hot path.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import, call or execute anything in this
package.  The product path (the CUDA library and its Python binding) never
imports it and shares no code with it; the only modules both sides use are the
seeded input generators in ``paper_1907_07774_gb300/synth.py``.

``fft``  -- plain recursive FFT and dense DFT (Sec. 3.3: 3D Fourier transforms).
``rd``   -- coefficients, Gaussian basis, Strang/CN forward, discrete adjoint,
            reduced gradient and Gauss-Newton Hessian-vector product.
"""
