"""Physical constants of the oracle (SI, IAU nominal values)."""
import math

C_SI = 299792458.0                     # speed of light [m/s]
GM_SUN_SI = 1.32712440018e20           # solar mass parameter [m^3/s^2]
MSUN_S = GM_SUN_SI / C_SI ** 3         # G M_sun / c^3 [s]
MPC_SI = 3.085677581491367e22          # megaparsec [m]
EULER_GAMMA = 0.5772156649015329
PI = math.pi
