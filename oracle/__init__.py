"""FP64 CPU oracle for the heterogeneous power-law attenuation FDTD method.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything here; the product
library never does, and it shares no code, header, table or helper with this
package.  Everything is written plainly from the paper (Sode & Pinton,
"Spatially heterogeneous power-law attenuation with multiple relaxation
mechanisms for ultrasound modeling"), in float64:

* ``fit``      -- power-law / Kramers-Kronig targets (Sec. 3.1, Eqs.
                  power_law_attenuation and kk_relation), the model complex
                  wavenumber (Sec. 2.2, Eqs. dispersion_relations / gamma1),
                  the normalised complex-wavenumber objective and the adaptive
                  Nelder-Mead calibration with the weight sweep (Sec. 3.2,
                  Table 2).
* ``medium``   -- per-voxel coefficient arrays in the paper's form (Sec. 2.1,
                  Eqs. relaxation_a / relaxation_b), PML inheritance and
                  profiles.
* ``stepper``  -- the staggered-grid time stepper (Sec. 2.1 Eqs. wave1, wave2,
                  relaxation4, relaxation_psi; Sec. 3.3), a plain C loop nest
                  in ``fw_oracle.c`` driven through ctypes.
* ``measure``  -- attenuation, dispersion and reflection measurements
                  (Sec. 4.1-4.3).
"""
