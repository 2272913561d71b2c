"""Seeded input generators shared by the oracle and the CUDA library.

This package writes the inputs that both paths read: the per-material
attenuation table file, voxel phantoms (uint8 material, FP16 density) and
source spectra.  It holds none of the transport, scoring, smoothing or
interpolation arithmetic of the method; the cross sections it tabulates are
the physics data the paper takes from Hubbell's tables (Sec. II-A), replaced
here by closed forms because those tables are not available.
"""

from .tables import (  # noqa: F401
    MATERIALS,
    Tables,
    build_tables,
    read_tables,
    write_tables,
    default_table_path,
)
from .phantoms import (  # noqa: F401
    cylinder_rod_phantom,
    cylinder_variant_phantom,
    ellipsoid_phantom,
    tiny_phantom,
    slab_phantom,
    fp16_bits,
    fp16_values,
)
from .spectrum import filtered_spectra, kramers_spectrum, mono_spectrum  # noqa: F401
from .detector import flat_panel_response, table_response  # noqa: F401
from .workloads import WORKLOADS, make_workload  # noqa: F401
