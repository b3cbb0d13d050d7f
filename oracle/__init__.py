"""FP64 CPU oracle for coronagraph wavefront propagation -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy implementations of what the CUDA path computes,
written from Douglas & Perrin, "Accelerated Modeling of Near and Far-Field Diffraction for
Coronagraphic Optical Systems" (SPIE 2018):

* ``optics``      -- sampling grid, optical elements (apertures, stops, thin lens, OPD
                     phasor of Eq. 3, Zernike, sine WFE, Gaussian-influence DM).
* ``fft``         -- textbook radix-2 Cooley-Tukey FFT (direct sums on the odd factor of N)
                     and the O(N^2) DFT sum.
* ``propagation`` -- centred DFT, angular-spectrum and direct Fresnel hops (Sec. 1.1,
                     Eq. 2), matrix Fourier transform (Sec. 1.1, Soummer et al. 2007).
* ``coronagraph`` -- semi-analytic Lyot chain, detector intensity and dark-hole sums.
* ``adjoint``     -- conjugate-transpose operators and the DM-height gradient.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference legs) may import this package. The product path never calls it: the library
fails loudly when its CUDA extension is missing instead of falling back to this code.

Every function computes in complex128 / float64 and is a direct transcription of a
definition (matmul serves as a step; the FFT is the textbook one of ``fft``; nothing is blocked
or fused).
"""
