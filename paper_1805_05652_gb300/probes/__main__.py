"""Build and run the arithmetic-rate probe (FP64 FMA, FP32 FMA, MUFU.EX2)."""

import os
import subprocess
import sys
import tempfile

from ..build import ARCH, nvcc

here = os.path.dirname(os.path.abspath(__file__))
exe = os.path.join(tempfile.gettempdir(), f"fmap_rates_{os.getpid()}")
subprocess.run([nvcc(), *ARCH, "-O3", "-o", exe, os.path.join(here, "rates.cu")], check=True)
sys.exit(subprocess.run([exe]).returncode)
