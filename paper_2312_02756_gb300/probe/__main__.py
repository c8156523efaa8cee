import json
import sys

from . import run

print(json.dumps(run(int(sys.argv[1]) if len(sys.argv) > 1 else 4096)))
